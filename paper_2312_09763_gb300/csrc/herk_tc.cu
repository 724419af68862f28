// herk_tc.cu -- Algorithm 2 step (v) of arXiv:2312.09763 (Sec. 3.1),
// V = Z Z^dagger (eq. "zz"), on the sm_103a tensor cores (tcgen05).
//
// Z is held as the real matrix U (rows 2(a n_feed + p) = Re Z, +1 = Im Z),
// split into two BF16 planes U = U_hi + U_lo.  Each CTA owns one 128 x 256
// tile of the lower triangle of G = U U^T and accumulates
//     G_tile += U_hi,i U_hi,j^T + U_hi,i U_lo,j^T + U_lo,i U_hi,j^T
// with tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM).  The
// accumulator is double-buffered in TMEM (2 x 256 columns): every
// `flush` k-blocks of 64 sources the MMA warp switches buffer and the eight
// epilogue warps add the finished buffer into FP32 running sums held in
// registers.  This bounds how many tensor-core accumulation steps any one
// FP32 partial sees, which keeps the summation error at FP32 level over
// 1e5 sources.  The epilogue folds 2 x 2 blocks of G into complex V:
//     Re V_ab = G[2a][2b] + G[2a+1][2b+1],   Im V_ab = G[2a+1][2b] - G[2a][2b+1].
//
// Roles (320 threads): warp 0 issues TMA loads (128B-swizzled K-major
// tiles of U_hi / U_lo into a 2-stage shared-memory ring), warp 1 owns TMEM
// and issues the MMAs from one thread, warps 2..9 drain TMEM.  Every
// mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// records MV device timeout in the status word, stops, lets in-flight
// copies and MMAs land, frees TMEM and returns.
#include <cuda.h>
#include "common.cuh"

namespace mv {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;                       // 16 KB
constexpr int B_BYTES = BN * BK * 2;                       // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // 96 KB
constexpr int NUM_THREADS = 320;
constexpr int TMEM_COLS = 512;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

// kind::f16 instruction descriptor: D = F32, A = B = BF16 (format 1) or FP16
// (format 0), both K-major, N = 256, M = 128.
constexpr uint32_t idesc_for(bool fp16) {
    return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the wait gave up (timeout or another role aborted).
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u) {
            if (*abort_flag) return false;
            const unsigned long long now = gtimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kTimeoutNs) {
                *abort_flag = 1;
                atomicCAS(err, 0, (int)kDevTimeout);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups
// 1024 B apart, descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// tcgen05.wait::ld, with the loaded registers as in/out operands so that no
// use of them can be scheduled ahead of the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
          "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
          "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
        :
        : "memory");
}

// lower-triangle tiles: row tile ti (128 rows), column tile tj (256 rows of U), tj <= ti / 2
__device__ __forceinline__ void tile_of(int idx, int& ti, int& tj) {
    int i = 0;
    while (idx >= i / 2 + 1) { idx -= i / 2 + 1; ++i; }
    ti = i;
    tj = idx;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
k_herk_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
          const Inst* __restrict__ inst, int inst0, LiveTables lt, int n_ax, uint32_t idesc, int fp16,
          const float* __restrict__ amax, float2* __restrict__ V, int N, int flush, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.y;
    const Inst in = inst[inst0 + slot];
    int ti, tj;
    tile_of(blockIdx.x, ti, tj);
    const long long K = (long long)lt.n_live[in.t] * n_ax;
    const int KB = (int)(((K + kKPad - 1) / kKPad * kKPad) / BK);
    const int n_chunks = (KB + flush - 1) / flush;

    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * STAGES + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * STAGES + 2 + b]); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull(b), 1); mbar_init(tempty(b), 8); }
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
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0) {
        if (lane == 0) {
            for (int it = 0; it < KB; ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!wait_bounded(empty(s), ph ^ 1u, abort_flag, err)) break;
                mbar_expect_tx(full(s), STAGE_BYTES);
                const uint32_t st = sbase + s * STAGE_BYTES;
                const int x = it * BK;
                tma_load_3d(st, &map_hi, x, ti * BM, slot, full(s));
                tma_load_3d(st + A_BYTES, &map_lo, x, ti * BM, slot, full(s));
                tma_load_3d(st + 2 * A_BYTES, &map_hi, x, tj * BN, slot, full(s));
                tma_load_3d(st + 2 * A_BYTES + B_BYTES / 2, &map_hi, x, tj * BN + BN / 2, slot, full(s));
                tma_load_3d(st + 2 * A_BYTES + B_BYTES, &map_lo, x, tj * BN, slot, full(s));
                tma_load_3d(st + 2 * A_BYTES + B_BYTES + B_BYTES / 2, &map_lo, x, tj * BN + BN / 2, slot, full(s));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int c = 0; c < n_chunks && ok; ++c) {
                const int buf = c & 1;
                const uint32_t ph = (uint32_t)(c >> 1) & 1u;
                if (!wait_bounded(tempty(buf), ph ^ 1u, abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                const int kb_end = min(KB, (c + 1) * flush);
                uint32_t acc = 0;
                for (; it < kb_end; ++it) {
                    const int s = it % STAGES;
                    const uint32_t sph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(full(s), sph, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t a_hi = sdesc(st + kk * 32);
                        const uint64_t a_lo = sdesc(st + A_BYTES + kk * 32);
                        const uint64_t b_hi = sdesc(st + 2 * A_BYTES + kk * 32);
                        const uint64_t b_lo = sdesc(st + 2 * A_BYTES + B_BYTES + kk * 32);
                        tc_mma(d, a_hi, b_hi, idesc, acc);
                        acc = 1;
                        tc_mma(d, a_hi, b_lo, idesc, 1);
                        tc_mma(d, a_lo, b_hi, idesc, 1);
                    }
                    tc_commit(empty(s));
                }
                tc_commit(tfull(buf));
            }
        }
    } else {
        // epilogue: warps 2..9; TMEM lane quadrant q, column half h
        const int q = warp & 3, h = (warp - 2) >> 2;
        float run[128];
#pragma unroll
        for (int i = 0; i < 128; ++i) run[i] = 0.f;
        bool ok = true;
        for (int c = 0; c < n_chunks; ++c) {
            const int buf = c & 1;
            const uint32_t ph = (uint32_t)(c >> 1) & 1u;
            if (!wait_bounded(tfull(buf), ph, abort_flag, err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + h * 128);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t r[32];
                tmem_ld32(ta + g * 32, r);
                tmem_wait_ld(r);
#pragma unroll
                for (int i = 0; i < 32; ++i) run[g * 32 + i] += __uint_as_float(r[i]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(buf));
        }
        if (ok && !*abort_flag) {
            const int r = ti * BM + q * 32 + lane;
            const int a = r >> 1;
            const bool even = (lane & 1) == 0;
            float2* Vb = V + in.v_off;
            const int c0 = tj * BN + h * 128;
            // undo the FP16 scaling 2^e of both operands: two exact power-of-two steps
            const float unscale = fp16 ? ldexpf(1.f, -fp16_scale_exp(amax[slot])) : 1.f;
#pragma unroll
            for (int jj = 0; jj < 64; ++jj) {
                const float x0 = run[2 * jj], x1 = run[2 * jj + 1];
                const float y0 = __shfl_xor_sync(0xffffffffu, x0, 1);
                const float y1 = __shfl_xor_sync(0xffffffffu, x1, 1);
                const float g00 = even ? x0 : y0, g01 = even ? x1 : y1;
                const float g10 = even ? y0 : x0, g11 = even ? y1 : x1;
                const int b = (c0 + 2 * jj) >> 1;
                if ((jj & 1) == (lane & 1) && a < N && b < N && a >= b) {
                    const float re = ((g00 + g11) * unscale) * unscale;
                    // autocorrelations are real: the tensor core rounds the two
                    // symmetric entries of G separately, so drop that residue
                    const float im = a == b ? 0.f : ((g10 - g01) * unscale) * unscale;
                    Vb[(long long)a * N + b] = make_float2(re, im);
                    if (a != b) Vb[(long long)b * N + a] = make_float2(re, -im);
                }
            }
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, long long k_pitch, int rows, int n_slots, bool fp16) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)k_pitch, (cuuint64_t)rows, (cuuint64_t)n_slots};
    cuuint64_t strides[2] = {(cuuint64_t)k_pitch * 2, (cuuint64_t)k_pitch * 2 * rows};
    cuuint32_t box[3] = {BK, BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool herk_tc_available() { return get_encode() != nullptr; }

cudaError_t launch_herk_tc(const Inst* d_inst, int inst0, int n_inst, LiveTables lt, int n_ax,
                           const __nv_bfloat16* d_hi, const __nv_bfloat16* d_lo, int rows, long long k_pitch,
                           int n_slots, int fp16, const float* d_amax, float2* d_v, int N, int flush, int* d_err,
                           cudaStream_t st, long long* launches) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_herk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    CUtensorMap mh, ml;
    if (!make_map(&mh, d_hi, k_pitch, rows, n_slots, fp16) || !make_map(&ml, d_lo, k_pitch, rows, n_slots, fp16))
        return cudaErrorInvalidValue;
    const int T = (rows + BM - 1) / BM;
    int n_tiles = 0;
    for (int i = 0; i < T; ++i) n_tiles += i / 2 + 1;
    if (flush < 1) flush = 4;
    dim3 grid(n_tiles, n_inst);
    k_herk_tc<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(mh, ml, d_inst, inst0, lt, n_ax, idesc_for(fp16 != 0), fp16,
                                                     d_amax, d_v, N, flush, d_err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
