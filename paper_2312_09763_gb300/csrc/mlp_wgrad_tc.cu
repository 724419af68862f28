// mlp_wgrad_tc.cu -- every weight gradient of a training batch of the learned
// beam in one launch on the sm_103a tensor cores.  For each product p (the
// output layer and the hidden layers)
//     dW_p = A_p^T X_p  and  db_p = A_p^T 1,
// A_p the layer's dL/dz (or dL/dy) and X_p its input, both [batch][width] as
// the training pass stores them, are summed over a range of the batch per
// k-split into FP32 partials (the optimiser adds the partials of every split
// in a fixed order).  A unit is (product, 128-row tile of A^T, k-split); one
// persistent CTA per SM walks them.  Both operands are read batch-major as
// MN-major tcgen05 operands (64-element boxes of 64 batch rows, 128-byte
// swizzle); warp 0 streams them by TMA through a ring of stages, warp 1 issues
// the MMAs (M = 128, N = the layer's input width, K = 16) and, per K step, one
// more MMA against a constant all-ones 16 x 64 tile whose result columns are
// the row sums of A^T (the bias gradient), and warps 2-17 write the partials.
// Every mbarrier wait is bounded (tc.cuh): on expiry the kernel records a
// device timeout, lets copies and MMAs in flight land, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include "common.cuh"
#include "tc.cuh"

namespace mv {
namespace {

using namespace tc;
typedef __nv_bfloat16 bf16;

constexpr int TM = 128;                  // rows of A^T per unit
constexpr int BK = 64;                   // batch rows per k-block
constexpr int MAXP = kWgradMaxProducts;
constexpr int A_BYTES = TM * BK * 2;     // 16 KB: two 64-row MN boxes
constexpr int B_BYTES = 256 * BK * 2;    // 32 KB: up to four
constexpr int STAGE = A_BYTES + B_BYTES;
constexpr int STAGES = 4;
constexpr int ONES = 16 * BK * 2;        // all-ones K-major tile, 2 KB
constexpr int EPI_WARPS = 16;            // four per TMEM lane quadrant, 64 columns each
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int TMEM_COLS = 512;           // accumulator [0, 256), row sums [256, 272)
constexpr int SMEM_BYTES = STAGES * STAGE + ONES + 256 + 1024;

struct Prod {
    int M, N;             // rows of A^T, columns of X (N <= 256)
    int m_tiles, unit0;   // 128-row tiles of A^T; first unit of this product
    int b_boxes;          // 64-column boxes of X per k-block
    float* out;           // partial s of (m, n) at out + s part_stride + m ldo + n
    long long ldo, part_stride;
    float* bias_part;     // partial s of the bias of row m at bias_part + s ldo_bias + m
    long long ldo_bias;
};
struct Job {
    int n_prod, splits, kblocks, n_units;
    Prod p[MAXP];
};
struct Maps {
    CUtensorMap a[MAXP], b[MAXP];
};
static_assert(sizeof(Maps) + sizeof(Job) + sizeof(int*) <= 4096, "kernel parameters over 4 KB");

// Shared-memory descriptor of an MN-major operand: 64-element MN boxes of 64 K
// rows (8 KB apart), 128-byte swizzle, groups of 8 K rows 1 KB apart.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct Unit {
    int prod, m0, kb0, kb1, split;
};

__device__ __forceinline__ Unit unit_at(const Job& j, int u) {
    Unit x;
    int p = 0;
    while (p + 1 < j.n_prod && j.p[p + 1].unit0 <= u) ++p;
    const int v = u - j.p[p].unit0;
    x.prod = p;
    x.split = v / j.p[p].m_tiles;
    x.m0 = (v % j.p[p].m_tiles) * TM;
    x.kb0 = (int)((long long)j.kblocks * x.split / j.splits);
    x.kb1 = (int)((long long)j.kblocks * (x.split + 1) / j.splits);
    return x;
}

__global__ void __launch_bounds__(THREADS, 1)
k_wgrad(const __grid_constant__ Maps maps, const __grid_constant__ Job j, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t ones = sbase + STAGES * STAGE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE + ONES);
    // full[STAGES], empty[STAGES], tfull, tempty
    const uint32_t b0 = smem_u32(bars);
    const uint32_t FULL = b0, EMPTY = b0 + 8u * STAGES, TFULL = b0 + 16u * STAGES, TEMPTY = TFULL + 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    {  // BF16 1.0 everywhere: the 128-byte swizzle permutes nothing that matters
        uint32_t* o = reinterpret_cast<uint32_t*>(smem + STAGES * STAGE);
        for (int i = threadIdx.x; i < ONES / 4; i += blockDim.x) o[i] = 0x3F803F80u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(FULL + 8u * s, 1); mbar_init(EMPTY + 8u * s, 1); }
        mbar_init(TFULL, 1);
        mbar_init(TEMPTY, EPI_WARPS);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < j.n_units && ok; u += gridDim.x) {
                const Unit x = unit_at(j, u);
                const Prod& P = j.p[x.prod];
                for (int kb = x.kb0; kb < x.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!wait_bounded_spin(EMPTY + 8u * s, ((uint32_t)(it / STAGES) & 1u) ^ 1u, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + s * STAGE;
                    mbar_expect_tx(FULL + 8u * s, (uint32_t)(A_BYTES + P.b_boxes * 8192));
                    // A^T rows [m0, m0 + 128) as two 64-row boxes (rows past M read zeros)
                    tma_load_2d(st, &maps.a[x.prod], x.m0, kb * BK, FULL + 8u * s);
                    tma_load_2d(st + A_BYTES / 2, &maps.a[x.prod], x.m0 + 64, kb * BK, FULL + 8u * s);
                    for (int b = 0; b < P.b_boxes; ++b)
                        tma_load_2d(st + A_BYTES + b * 8192, &maps.b[x.prod], 64 * b, kb * BK, FULL + 8u * s);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, cnt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < j.n_units && ok; u += gridDim.x, ++cnt) {
                const Unit x = unit_at(j, u);
                const int ncols = (j.p[x.prod].N + 15) / 16 * 16;
                if (!wait_bounded_spin(TEMPTY, ((uint32_t)cnt & 1u) ^ 1u, abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                // both operands MN-major: bits 15 (A) and 16 (B)
                const uint32_t id = idesc_f16(false, TM, ncols) | (1u << 15) | (1u << 16);
                const uint32_t id_ones = idesc_f16(false, TM, 16) | (1u << 15);
                for (int kb = x.kb0; kb < x.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!wait_bounded_spin(FULL + 8u * s, (uint32_t)(it / STAGES) & 1u, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t acc = (kb > x.kb0 || kk > 0) ? 1u : 0u;
                        // K step kk: 16 batch rows (2 KB) into every MN box
                        tc_mma(tmem, sdesc_mn(st + kk * 2048), sdesc_mn(st + A_BYTES + kk * 2048), id, acc);
                        tc_mma(tmem + 256u, sdesc_mn(st + kk * 2048), sdesc(ones), id_ones, acc);
                    }
                    tc_commit(EMPTY + 8u * s);
                }
                if (!ok) break;
                tc_commit(TFULL);
            }
        }
    } else {
        // epilogue: TMEM lane quadrant q (rows 32 q .. 32 q + 31 of the tile),
        // columns [64 cq, 64 cq + 64)
        const int q = warp & 3, cq = (warp - 2) >> 2;
        int cnt = 0;
        for (int u = blockIdx.x; u < j.n_units; u += gridDim.x, ++cnt) {
            const Unit x = unit_at(j, u);
            const Prod& P = j.p[x.prod];
            if (!wait_bounded_spin(TFULL, (uint32_t)cnt & 1u, abort_flag, err)) break;
            tc_fence_after();
            const int m = x.m0 + q * 32 + lane;
            const bool valid = m < P.M;
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16);
            const int ncols = (P.N + 15) / 16 * 16;
            float* o = P.out + (long long)x.split * P.part_stride + (long long)m * P.ldo;
            for (int c0 = cq * 64; c0 < min(ncols, cq * 64 + 64); c0 += 32) {
                uint32_t r[32];
                tmem_ld32(ta + c0, r);
                tmem_wait_ld(r);
                const int nv = min(32, P.N - c0);
                if (valid) {
                    if (nv == 32) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            *reinterpret_cast<float4*>(o + c0 + 4 * i) =
                                make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                            __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3]));
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (i < nv) o[c0 + i] = __uint_as_float(r[i]);
                    }
                }
            }
            if (cq == 0) {  // row sums of A^T (any of the 16 equal columns)
                uint32_t r[16];
                tmem_ld16(ta + 256u, r);
                tmem_wait_ld16(r);
                if (valid) P.bias_part[(long long)x.split * P.ldo_bias + m] = __uint_as_float(r[0]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(TEMPTY);
            if (*abort_flag) break;
        }
    }
    __syncthreads();
    if (*abort_flag) {
        // let copies and MMAs already issued land before TMEM and smem go away
        const unsigned long long t0 = gtimer();
        while (gtimer() - t0 < 2000000ull) {}
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// MN-major operand [kext][ld] (rows contiguous): dims (rows, kext), boxes of
// 64 rows x 64 batch rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const bf16* p, long long ld, int rows, long long kext) {
    EncodeTiledFn enc = get_encode();
    if (!enc || ((uintptr_t)p & 15) || (ld * 2) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)kext};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, BK};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(p), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t wgrad_tc_init() {
    return cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t launch_wgrad_tc(const WgradProduct* p, int n_prod, long long kext, int splits, int n_sms, int* d_err,
                            cudaStream_t st, long long* launches) {
    if (n_prod < 1 || n_prod > MAXP || kext < BK || splits < 1) return cudaErrorInvalidValue;
    Maps maps{};
    Job j{};
    j.n_prod = n_prod;
    j.kblocks = (int)((kext + BK - 1) / BK);
    j.splits = std::min(splits, j.kblocks);
    int units = 0;
    for (int i = 0; i < n_prod; ++i) {
        const WgradProduct& w = p[i];
        // A^T rows and X columns: at least one 64-row box each, X at most 256 wide
        if (w.M < 1 || w.a_rows < 64 || w.M > w.a_rows || w.N < 1 || w.N > 256 || w.b_rows < 64 ||
            w.N > w.b_rows || w.lda < w.a_rows || w.ldb < w.b_rows)
            return cudaErrorInvalidValue;
        if (!make_map(&maps.a[i], w.A, w.lda, w.a_rows, kext) || !make_map(&maps.b[i], w.X, w.ldb, w.b_rows, kext))
            return cudaErrorInvalidValue;
        Prod& P = j.p[i];
        P.M = w.M;
        P.N = w.N;
        P.m_tiles = (w.M + TM - 1) / TM;
        P.unit0 = units;
        P.b_boxes = (w.N + 63) / 64;
        P.out = w.out;
        P.ldo = w.ldo;
        P.part_stride = w.part_stride;
        P.bias_part = w.bias_part;
        P.ldo_bias = w.ldo_bias;
        units += P.m_tiles * j.splits;
    }
    j.n_units = units;
    const int grid = std::max(1, std::min(n_sms, units));
    k_wgrad<<<grid, THREADS, SMEM_BYTES, st>>>(maps, j, d_err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
