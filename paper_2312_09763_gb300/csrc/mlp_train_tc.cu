// mlp_train_tc.cu -- the learned beam's network one matrix product per launch
// on the sm_103a tensor cores: its batched evaluation, and the training of
// network shapes that the fused training pass (mlp_chain_tc.cu) and the
// one-launch weight gradients (mlp_wgrad_tc.cu) do not cover.
//
// Every product of the network's forward and backward pass is written as
//     D[M][N] = A[M][K] B[N][K]^T
// with BF16 operands in global memory, K-major ([rows][K]: the forward and
// input-gradient products, with the weights and their transposed copies
// that the optimiser writes) or MN-major ([K][rows]: the weight gradients
// dW = dZ^T X read dZ and X as the batch-major arrays the other products
// write, with no transposed copies).  In shared memory a K-major operand is
// one 64-column, 128-byte-swizzled box per 64 K; an MN-major one is 64-element
// MN boxes of 64 K rows (8 KB each, 128-byte swizzle), the MMA descriptor
// stepping 8 KB between MN boxes and 1 KB between groups of 8 K rows.  One
// persistent CTA per SM walks units (row tile, up-to-256-column tile,
// k-split) in a fixed order; warp 0 streams 64-K panels of A and B (up to
// 256 rows) with TMA through a ring of stages, warp 1 owns TMEM and issues tcgen05.mma (M = 128, N = the
// tile's width, K = 16; FP32 accumulation), and warps 2-17 (four per TMEM
// lane quadrant, one output row per thread) drain the accumulators through
// the fused epilogue of the product:
//   RELU  h = relu(acc + b)             -> BF16 rows, and BF16 columns (transpose)
//   LOSS  y = acc + b, r = y - target   -> dL/dy = g r in BF16 rows and columns,
//                                          sum of r^2 into the loss
//   MASK  dz = acc * (h_prev > 0)        -> BF16 rows and columns (ReLU derivative)
//   F32   acc                            -> FP32 partial of k-split s (weight gradients)
//   EMB   acc                            -> added into the embedding gradient of the
//                                          row's beam
//   Y     acc + b                        -> FP32 outputs (evaluation)
// A weight-gradient product dW = dZ^T X (F32 with bias_part) also yields the
// bias gradient, the row sums of its A operand dZ^T: one more MMA per K step
// against a constant all-ones 16 x 64 tile in shared memory (N = 16, one
// sixteenth of the main MMA's work) accumulates them in TMEM columns
// [256, 272), and the epilogue writes one partial per k-split.
//
// Row tiles are 128 rows with two TMEM accumulators (the epilogue of one
// unit overlaps the MMAs of the next), or, for the weight-gradient products
// whose K axis (the batch) is long and whose output is small, 256 rows: two
// 128-row MMAs share every B panel, accumulators at TMEM columns 0 and 256.
// Every mbarrier wait is bounded (tc.cuh) and spins (these kernels are
// short: a hinted sleep can outlast the wait): on expiry the kernel records a
// device timeout, lets in-flight copies and MMAs land, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include "common.cuh"
#include "tc.cuh"

namespace mv {
namespace {

using namespace tc;
typedef __nv_bfloat16 bf16;

constexpr int TM = 128;                       // rows per MMA
constexpr int BK = 64;                        // K columns per panel (128 bytes of BF16)
constexpr int BMAX = 256;                     // B rows per tile at most
constexpr int A_BYTES = TM * BK * 2;          // 16 KB per 128-row A box
constexpr int B_BYTES_MAX = BMAX * BK * 2;    // 32 KB
constexpr int RING = 192 * 1024;              // 4 stages of 48 KB, or 3 of 64 KB (two A boxes)
constexpr int MAX_STAGES = 4;
constexpr int EPI_WARPS = 16;                 // four per TMEM lane quadrant
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int TMEM_COLS = 512;
constexpr int ONES = 16 * BK * 2;             // all-ones B tile for the row sums (2 KB)
constexpr int SMEM_BYTES = RING + ONES + 256 + 1024;

struct Job {
    int M, N;               // valid output rows and columns
    int mt;                 // 128-row MMAs per unit (1 or 2)
    int m_tiles, n_tiles, splits, kblocks;
    int bnb;                // B rows per tile (the B tensor map's box)
    int stages, stage_bytes;
    int ones;               // row sums of A in TMEM columns [256, 272) (single accumulator)
    int a_mn, b_mn;         // operand layouts (1: MN-major)
    GemmEpi e;
};

// Shared-memory descriptor of an MN-major operand: 64-element MN boxes of 64 K
// rows (8 KB apart), 128-byte swizzle, groups of 8 K rows 1 KB apart.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void st_global_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Sum of x over the warp's 32 lanes, for 32 columns at once: after the
// butterfly lane l holds the sum of column l (31 shuffles).
__device__ __forceinline__ float column_sums(float (&x)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = up ? x[i] : x[i + w];
            const float keep = up ? x[i + w] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return x[0];
}

struct UnitPos {
    int m0, n0, ncols, kb0, kb1, split;
};

__device__ __forceinline__ UnitPos unit_pos(const Job& j, int u) {
    UnitPos p;
    const int tiles = j.m_tiles * j.n_tiles;
    p.split = u / tiles;
    const int t = u % tiles;
    p.m0 = (t % j.m_tiles) * TM * j.mt;
    const int nt = t / j.m_tiles;
    p.n0 = nt * j.bnb;
    p.ncols = min(j.bnb, (j.N - p.n0 + 15) / 16 * 16);
    p.kb0 = (int)((long long)j.kblocks * p.split / j.splits);
    p.kb1 = (int)((long long)j.kblocks * (p.split + 1) / j.splits);
    return p;
}

// KIND: the epilogue (GemmEpiKind), a compile-time constant so that each
// product carries only its own epilogue's registers.
template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
          const __grid_constant__ Job j, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // barriers: full[MAX_STAGES], empty[MAX_STAGES], tfull[2], tempty[2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING + ONES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MAX_STAGES + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = j.stages, SB = j.stage_bytes, MT = j.mt;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[MAX_STAGES + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * MAX_STAGES + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * MAX_STAGES + 2 + b]); };
    if (j.ones) {  // BF16 1.0 everywhere: the 128-byte swizzle permutes nothing that matters
        uint32_t* o = reinterpret_cast<uint32_t*>(smem + RING);
        for (int i = threadIdx.x; i < ONES / 4; i += blockDim.x) o[i] = 0x3F803F80u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull(b), 1); mbar_init(tempty(b), EPI_WARPS); }
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
    const uint32_t sbase = smem_u32(smem);
    const int n_units = j.m_tiles * j.n_tiles * j.splits;
    const int b_boxes = (j.bnb + 63) / 64;  // MN-major B: 64-element boxes (the last may read past N as zeros)
    const uint32_t tx_bytes = (uint32_t)(MT * A_BYTES + (j.b_mn ? b_boxes * 8192 : j.bnb * BK * 2));
    // one accumulator set per unit with two 128-row MMAs or the row sums;
    // else two sets in turn
    const bool single = MT == 2 || j.ones;
    auto buf_of = [&](int cnt) { return single ? 0 : cnt & 1; };
    auto phase_of = [&](int cnt) { return single ? (uint32_t)cnt & 1u : (uint32_t)(cnt >> 1) & 1u; };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const UnitPos p = unit_pos(j, u);
                for (int kb = p.kb0; kb < p.kb1; ++kb, ++it) {
                    const int s = it % S;
                    if (!wait_bounded_spin(empty(s), ((uint32_t)(it / S) & 1u) ^ 1u, abort_flag, err)) { ok = false; break; }
                    mbar_expect_tx(full(s), tx_bytes);
                    const uint32_t st = sbase + s * SB;
                    for (int t = 0; t < MT; ++t) {
                        if (j.a_mn) {  // two 64-row MN boxes per 128-row tile
                            tma_load_2d(st + t * A_BYTES, &map_a, p.m0 + t * TM, kb * BK, full(s));
                            tma_load_2d(st + t * A_BYTES + A_BYTES / 2, &map_a, p.m0 + t * TM + 64, kb * BK, full(s));
                        } else {
                            tma_load_2d(st + t * A_BYTES, &map_a, kb * BK, p.m0 + t * TM, full(s));
                        }
                    }
                    if (j.b_mn) {
                        for (int b = 0; b < b_boxes; ++b)
                            tma_load_2d(st + MT * A_BYTES + b * 8192, &map_b, p.n0 + 64 * b, kb * BK, full(s));
                    } else {
                        tma_load_2d(st + MT * A_BYTES, &map_b, kb * BK, p.n0, full(s));
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, cnt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++cnt) {
                const UnitPos p = unit_pos(j, u);
                const int buf = buf_of(cnt);
                if (!wait_bounded_spin(tempty(buf), phase_of(cnt) ^ 1u, abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                // operand majors: bit 15 (A), bit 16 (B) set for MN-major
                const uint32_t id = idesc_f16(false, TM, p.ncols) | ((uint32_t)j.a_mn << 15) | ((uint32_t)j.b_mn << 16);
                const uint32_t id_ones = idesc_f16(false, TM, 16) | ((uint32_t)j.a_mn << 15);
                for (int kb = p.kb0; kb < p.kb1; ++kb, ++it) {
                    const int s = it % S;
                    if (!wait_bounded_spin(full(s), (uint32_t)(it / S) & 1u, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = sbase + s * SB;
                    // K step kk: 32 bytes into every K-major row, or 16 K rows (2 KB) of
                    // every MN-major box
                    auto adesc = [&](int t, int kk) {
                        const uint32_t a = st + t * A_BYTES;
                        return j.a_mn ? sdesc_mn(a + kk * 2048) : sdesc(a + kk * 32);
                    };
                    const uint32_t b = st + MT * A_BYTES;
                    for (int t = 0; t < MT; ++t) {
                        const uint32_t d = tmem + (uint32_t)((MT == 2 ? t : buf) * 256);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            tc_mma(d, adesc(t, kk), j.b_mn ? sdesc_mn(b + kk * 2048) : sdesc(b + kk * 32), id,
                                   (kb > p.kb0 || kk > 0) ? 1u : 0u);
                    }
                    if (j.ones) {
                        // row sums of A: A times the all-ones tile (K-major), N = 16
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            tc_mma(tmem + 256u, adesc(0, kk), sdesc(sbase + RING), id_ones, (kb > p.kb0 || kk > 0) ? 1u : 0u);
                    }
                    tc_commit(empty(s));
                }
                if (!ok) break;
                tc_commit(tfull(buf));
            }
        }
    } else {
        // epilogue warp: TMEM lane quadrant q4, one output row per thread, and
        // its share of the unit's columns: a quarter of the tile (one 128-row
        // MMA) or half of one of the two 128-row halves (two)
        const int q4 = warp & 3, cq = (warp - 2) >> 2;
        const int half = MT == 2 ? cq >> 1 : 0;
        const int cw = MT == 2 ? 128 : 64;
        const int cbeg = MT == 2 ? (cq & 1) * 128 : cq * 64;
        const GemmEpi& e = j.e;
        int cnt = 0;
        for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++cnt) {
            const UnitPos p = unit_pos(j, u);
            const int buf = buf_of(cnt);
            if (!wait_bounded_spin(tfull(buf), phase_of(cnt), abort_flag, err)) break;
            tc_fence_after();
            const int m = p.m0 + half * TM + q4 * 32 + lane;
            const bool valid = m < j.M;
            const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((MT == 2 ? half : buf) * 256);
            float lsum = 0.f;
            for (int c0 = cbeg; c0 < min(p.ncols, cbeg + cw); c0 += 32) {
                uint32_t r[32];
                tmem_ld32(ta + c0, r);
                tmem_wait_ld(r);
                const int n0 = p.n0 + c0;
                const int nv = min(32, j.N - n0);  // valid columns of this chunk
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
                if constexpr (KIND == GEPI_RELU || KIND == GEPI_MASK) {
                    if constexpr (KIND == GEPI_RELU) {
                        if (nv == 32) {  // bias rows are 32-byte aligned
                            const float4* b4 = reinterpret_cast<const float4*>(e.bias + n0);
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 b = __ldg(b4 + q);
                                v[4 * q] = fmaxf(v[4 * q] + b.x, 0.f);
                                v[4 * q + 1] = fmaxf(v[4 * q + 1] + b.y, 0.f);
                                v[4 * q + 2] = fmaxf(v[4 * q + 2] + b.z, 0.f);
                                v[4 * q + 3] = fmaxf(v[4 * q + 3] + b.w, 0.f);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] = i < nv ? fmaxf(v[i] + e.bias[n0 + i], 0.f) : 0.f;
                        }
                    } else {
                        if (valid && nv == 32) {  // 64 bytes of the mask row, 16-byte aligned
                            const bf16* mk = e.mask + (long long)m * e.ldm + n0;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint4 w = __ldg(reinterpret_cast<const uint4*>(mk) + q);
                                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    // a ReLU output is positive exactly when its BF16 bits,
                                    // read as a signed 16-bit integer, are
                                    v[8 * q + 2 * h] = (short)(ww[h] & 0xFFFFu) > 0 ? v[8 * q + 2 * h] : 0.f;
                                    v[8 * q + 2 * h + 1] = (short)(ww[h] >> 16) > 0 ? v[8 * q + 2 * h + 1] : 0.f;
                                }
                            }
                        } else if (valid) {
                            const bf16* mk = e.mask + (long long)m * e.ldm + n0;
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                v[i] = (i < nv && __bfloat162float(mk[i]) > 0.f) ? v[i] : 0.f;
                        }
                        if (!valid) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] = 0.f;
                        }
                    }
                    if (valid) {
                        bf16* o = static_cast<bf16*>(e.out) + (long long)m * e.ldo + n0;
                        if (nv == 32) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                st_global_v4(o + 8 * q, pack2(v[8 * q], v[8 * q + 1]), pack2(v[8 * q + 2], v[8 * q + 3]),
                                             pack2(v[8 * q + 4], v[8 * q + 5]), pack2(v[8 * q + 6], v[8 * q + 7]));
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (i < nv) o[i] = __float2bfloat16(v[i]);
                        }
                        if (e.outT) {
                            // column n of the output is row n of the transpose: the
                            // warp's 32 rows land in 64 contiguous bytes
                            bf16* t = e.outT + (long long)n0 * e.ldt + m;
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (i < nv) t[(long long)i * e.ldt] = __float2bfloat16(v[i]);
                        }
                    }
                } else if constexpr (KIND == GEPI_LOSS) {
                    // columns [0, 16): network outputs n < n_out, zero gradient past them
                    float g[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        g[i] = 0.f;
                        if (valid && i < e.n_out) {
                            const float rr = v[i] + e.bias[i] - e.target[(long long)m * e.n_out + i];
                            lsum += rr * rr;
                            g[i] = e.gscale * rr;
                        }
                    }
                    if (valid) {
                        bf16* o = static_cast<bf16*>(e.out) + (long long)m * e.ldo;
                        st_global_v4(o, pack2(g[0], g[1]), pack2(g[2], g[3]), pack2(g[4], g[5]), pack2(g[6], g[7]));
                        st_global_v4(o + 8, pack2(g[8], g[9]), pack2(g[10], g[11]), pack2(g[12], g[13]),
                                     pack2(g[14], g[15]));
                        if (e.outT) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) e.outT[(long long)i * e.ldt + m] = __float2bfloat16(g[i]);
                        }
                    }
                } else if constexpr (KIND == GEPI_F32 || KIND == GEPI_Y) {
                    if (valid) {
                        float* o = static_cast<float*>(e.out) + (long long)p.split * e.part_stride + (long long)m * e.ldo + n0;
                        if constexpr (KIND == GEPI_Y) {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                if (i < nv && i < e.n_out) o[i] = v[i] + e.bias[n0 + i];
                        } else if (nv == 32) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                *reinterpret_cast<float4*>(o + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (i < nv) o[i] = v[i];
                        }
                    }
                } else if constexpr (KIND == GEPI_EMB) {
                    // rows of one beam summed over the warp before the atomic add (the
                    // training batch holds each beam's rows together)
                    const int a = valid ? e.ant[m] : -1;
                    unsigned rem = __ballot_sync(0xffffffffu, valid);
                    while (rem) {
                        const int al = __shfl_sync(0xffffffffu, a, __ffs(rem) - 1);
                        const unsigned grp = __ballot_sync(0xffffffffu, a == al);
                        float x[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) x[i] = a == al ? v[i] : 0.f;
                        const float cs = column_sums(x, lane);
                        if (lane < nv && n0 + lane < e.emb) atomicAdd(e.gemb + (long long)al * e.emb + n0 + lane, cs);
                        rem &= ~grp;
                    }
                }
            }
            if (KIND == GEPI_F32 && j.ones && cq == 0) {
                // row sums of A (any of the 16 equal columns)
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + 256u, r);
                tmem_wait_ld16(r);
                if (valid) e.bias_part[(long long)p.split * e.ldo_bias + m] = __uint_as_float(r[0]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(buf));
            if constexpr (KIND == GEPI_LOSS) {
                for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
                if (lane == 0 && lsum != 0.f) atomicAdd(e.loss, (double)lsum);
            }
            if (*abort_flag) break;
        }
    }
    __syncthreads();
    if (*abort_flag) {
        const unsigned long long t0 = gtimer();
        while (gtimer() - t0 < 2000000ull) {}
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

bool make_map(CUtensorMap* map, const GemmOperand& o, int box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    // K-major: (K, rows) with boxes of 64 K x box_rows rows; MN-major: (rows,
    // K) with boxes of 64 rows x 64 K
    cuuint64_t dims[2] = {(cuuint64_t)(o.mn ? o.rows : o.kext), (cuuint64_t)(o.mn ? o.kext : o.rows)};
    cuuint64_t strides[1] = {(cuuint64_t)o.ld * 2};
    cuuint32_t box[2] = {BK, (cuuint32_t)(o.mn ? BK : box_rows)};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(o.p), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t gemm_tc_init() {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)k_gemm_tc<GEPI_RELU>, (const void*)k_gemm_tc<GEPI_LOSS>,
                          (const void*)k_gemm_tc<GEPI_MASK>, (const void*)k_gemm_tc<GEPI_F32>,
                          (const void*)k_gemm_tc<GEPI_EMB>, (const void*)k_gemm_tc<GEPI_Y>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    return e;
}

int gemm_tc_grid(int M, int N, int splits, bool two_row_tiles, int kext, int n_sms) {
    const int mt = two_row_tiles ? 2 : 1;
    const int bnb = std::min(BMAX, (N + 15) / 16 * 16);
    const int kblocks = (kext + BK - 1) / BK;
    const int units = ((M + TM * mt - 1) / (TM * mt)) * ((N + bnb - 1) / bnb) * std::max(1, std::min(splits, kblocks));
    return std::max(1, std::min(n_sms, units));
}

cudaError_t launch_gemm_tc(const GemmOperand& A, const GemmOperand& B, int M, int N, int splits, bool two_row_tiles,
                           const GemmEpi& e, int n_sms, int* d_err, cudaStream_t st, long long* launches) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // operand shapes the TMA boxes need: K extents of one panel or more, A at
    // least one 128-row box, B at least as many rows as its box; 16-byte rows.
    // Row sums of A (bias_part) ride on weight-gradient products (F32, 128-row units).
    // K-major: A at least one 128-row box, B at least as many rows as its box,
    // K at least one 64-column panel.  MN-major: rows and K at least one 64 box
    // each (a 128-row A tile reads two MN boxes, the second may lie past the
    // rows and reads zeros), B's last box likewise.
    const int bnb = std::min(BMAX, (N + 15) / 16 * 16);
    auto bad = [&](const GemmOperand& o, bool is_a) {
        if (o.kext < BK || o.ld % 8 || ((uintptr_t)o.p & 15)) return true;
        if (o.mn) return o.rows < BK || o.ld < o.rows;
        return o.ld < o.kext || (is_a ? o.rows < TM : o.rows < bnb);
    };
    if (bad(A, true) || bad(B, false) || A.kext != B.kext || (B.mn && two_row_tiles) ||
        (A.mn && two_row_tiles) || (e.bias_part && (e.kind != GEPI_F32 || two_row_tiles)))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, TM) || !make_map(&mb, B, bnb)) return cudaErrorInvalidValue;
    Job j{};
    j.M = M;
    j.N = N;
    j.bnb = bnb;
    j.mt = two_row_tiles ? 2 : 1;
    j.stage_bytes = j.mt * A_BYTES + B_BYTES_MAX;
    j.stages = std::min(MAX_STAGES, RING / j.stage_bytes);
    j.m_tiles = (M + TM * j.mt - 1) / (TM * j.mt);
    j.n_tiles = (N + bnb - 1) / bnb;
    j.kblocks = (A.kext + BK - 1) / BK;
    j.splits = std::max(1, std::min(splits, j.kblocks));
    j.ones = e.bias_part != nullptr;
    j.a_mn = A.mn;
    j.b_mn = B.mn;
    j.e = e;
    const int grid = gemm_tc_grid(M, N, splits, two_row_tiles, A.kext, n_sms);
    switch (e.kind) {
        case GEPI_RELU: k_gemm_tc<GEPI_RELU><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        case GEPI_LOSS: k_gemm_tc<GEPI_LOSS><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        case GEPI_MASK: k_gemm_tc<GEPI_MASK><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        case GEPI_F32: k_gemm_tc<GEPI_F32><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        case GEPI_EMB: k_gemm_tc<GEPI_EMB><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        case GEPI_Y: k_gemm_tc<GEPI_Y><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, j, d_err); break;
        default: return cudaErrorInvalidValue;
    }
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
