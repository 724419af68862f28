// herk_tc.cu -- Algorithm 2 step (v) of arXiv:2312.09763 (Sec. 3.1),
// V = Z Z^dagger (eq. "zz"), on the sm_103a tensor cores (tcgen05).
//
// Z is held as the real matrix U (rows 2(a n_feed + p) = Re Z, +1 = Im Z),
// scaled by an exact power of two into FP16 range and split into two FP16
// planes U = U_hi + U_lo.  A persistent kernel (one CTA per SM) takes units of
// work (instance, 128 x BN tile of the lower triangle of G = U U^T, k-range)
// from an atomic counter and accumulates
//     G_tile += U_hi,i U_hi,j^T + U_hi,i U_lo,j^T + U_lo,i U_hi,j^T
// with tcgen05.mma (kind::f16, FP32 accumulate in TMEM, BN = 128 or 256).
// The accumulator is double-buffered in TMEM: every `flush` k-blocks of 64
// sources the MMA warp switches buffer and the epilogue warps add the
// finished buffer into FP32 running sums (registers, or TMEM in the fused
// variant).  This bounds how many tensor-core accumulation steps any one
// FP32 partial sees, which keeps the summation error at FP32 level over 1e5
// sources.  The epilogue folds 2 x 2 blocks of G into complex V:
//     Re V_ab = G[2a][2b] + G[2a+1][2b+1],   Im V_ab = G[2a+1][2b] - G[2a][2b+1],
// or writes raw partial tiles when the k-range is split (k_herk_finalize
// sums them).
//
// Roles: warp 0 fetches units and issues TMA loads (128B-swizzled K-major
// tiles of U_hi / U_lo into a shared-memory ring), warp 1 owns TMEM and
// issues the MMAs from one thread, BN / 32 warps drain TMEM, and in the
// fused variant further warps build the next batch's U (zcore.cuh).  Every
// mbarrier wait is bounded (tc.cuh); on expiry the kernel records MV device
// timeout in the status word, stops, lets in-flight copies and MMAs land,
// frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <type_traits>
#include "common.cuh"
#include "tc.cuh"
#include "zcore.cuh"

namespace mv {
namespace {

using namespace tc;

constexpr int BM = 128;  // tile rows

// k-block of a tile width: 64 sources (128-byte rows, 128-byte swizzle) for
// 128-column tiles, 32 sources (64-byte rows, 64-byte swizzle) for 256-column
// tiles, whose ring then holds four stages instead of two: the same 192 KB in
// finer steps, so more of it is in flight while the MMAs read one stage.
template <int BN>
__host__ __device__ constexpr int bk_for() { return BN == 256 ? 32 : 64; }

// Shared-memory descriptor of a K-major operand tile with rows of BK 16-bit
// elements: 8-row groups 8 BK 2 bytes apart, swizzle of the row width.
template <int BK>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
    static_assert(BK == 64 || BK == 32, "128- or 64-byte rows");
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * BK * 2) >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)(BK == 64 ? 2 : 4) << 61);
}
// ------------------------------------------------------------------ tiling
// Lower-triangle tiles of G, row panel by row panel: panel ti (rows [ti BM,
// ti BM + BM)) needs the columns [0, cmax), taken BN at a time.  With
// 256-column tiles cmax = min(BM (ti + 1), rows rounded up to 16), so the last
// chunk of a panel (the one holding the diagonal) is cmax - c0 wide, a
// multiple of 16 (the MMA's N): at 700 rows 12 tiles, four of them 128 wide
// and one 192 (336 K of executed area for the 245 K of the triangle, against
// 393 K for full tiles).  128-column tiles stay full (cmax = BM (ti + 1)): a
// 64-wide MMA tile costs as much as a full one.  Tile index runs over the
// chunks in row order.
template <int BN>
__host__ __device__ __forceinline__ int panel_cmax(int ti, int rows) {
    return BN == 128 ? BM * (ti + 1) : min(BM * (ti + 1), (rows + 15) / 16 * 16);
}

template <int BN>
__host__ __device__ __forceinline__ void tile_at(int idx, int rows, int& ti, int& c0, int& ncol) {
    if constexpr (BN == 128) {  // panel i holds i + 1 full tiles
        int i = 0;
        while (idx > i) idx -= ++i;
        ti = i;
        c0 = idx * BN;
        ncol = BN;
    } else {
        for (int i = 0;; ++i) {
            const int cmax = panel_cmax<BN>(i, rows), nch = (cmax + BN - 1) / BN;
            if (idx < nch) {
                ti = i;
                c0 = idx * BN;
                ncol = min(BN, cmax - c0);
                return;
            }
            idx -= nch;
        }
    }
}

template <int BN>
int n_tiles_for(int rows) {
    const int T = (rows + BM - 1) / BM;
    int n = 0;
    for (int i = 0; i < T; ++i) n += (panel_cmax<BN>(i, rows) + BN - 1) / BN;
    return n;
}

// Kernel-wide configuration for a tile width BN (128 or 256 columns); ZW > 0:
// the kernel also runs the Z build of the next batch on ZW extra warps, and
// keeps the epilogue's running sums in TMEM so that registers are free for
// them: at 128 columns two accumulators [0, 256) and the sums [256, 384); at
// 256 columns one accumulator [0, 256) and the sums [256, 512), the MMAs
// waiting while the epilogue adds a finished chunk into the sums (SB).
template <int BN, int ZW = 0>
struct Cfg {
    static constexpr bool FZ = ZW > 0;
    static constexpr bool SB = FZ && BN == 256;                    // single accumulator buffer
    static constexpr int RUN = SB ? BN : 2 * BN;                   // TMEM column of the running sums
    static constexpr int BK = bk_for<BN>();
    static constexpr int SUB = BM * BK * 2;                        // one 128-row box of one plane
    static constexpr int A_BYTES = SUB;                            // 16 or 8 KB per plane
    static constexpr int B_BYTES = BN * BK * 2;                    // 16 KB per plane either way
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 64 or 48 KB
    static constexpr int STAGES = BN == 256 ? 4 : 3;               // 192 KB of ring either way
    static constexpr int TMEM_COLS = (BN == 256 || FZ) ? 512 : 256;  // two accumulators (+ running sums)
    static constexpr int EPI_WARPS = BN / 32;                      // 128 columns per epilogue warp
    static constexpr int Z_WARPS = ZW;
    static constexpr int THREADS = (2 + EPI_WARPS + Z_WARPS) * 32;
    static constexpr int QDEPTH = 4;                               // unit-id queue depth
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512 + Z_WARPS * 16 * 4;
};

// Z-build warps of a fused HERK: 6, with 12 warps in all (3 per SM
// sub-partition, up to 168 registers a thread, so the Z build keeps its WA
// prefetch).  On the 350-antenna workload a sweep of 4 to 14 warps was
// fastest at 6-7: more warps slow the tensor pipe's feed, fewer leave the Z
// build behind.
__host__ __device__ constexpr int zwarps(int zp, int za, int zf) { return zp == 0 || za * zf == 0 ? 0 : 6; }

// kind::f16 instruction descriptor: D = F32, A = B = BF16 (format 1) or FP16
// (format 0), both K-major, N = BN, M = 128.
constexpr uint32_t idesc_for(bool fp16, int bn) {
    return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

// One unit of work: instance slot, tile (ti, tj) and the k-block range
// [kb0, kb1) of split ks of S (balanced integer split of the instance's K).
// Unit u = (r S + ks) n_tiles + tile, where r ranks the batch's instances by
// decreasing live count (order[r] = slot): the longest instances are fetched
// first, and the CTAs running at one time share k-ranges of one instance, so
// each 64-column block of U is read from HBM about once and reused via L2.
struct Unit {
    int slot, r0, c0, ncol, kb0, kb1;  // first A row, first B row and width of the tile
    int rlim, clim;                    // rows / columns past these belong to no block
    int part;  // index of the unit's partial tile: (slot n_tiles + tile) S + ks
};

// 128-row boxes of U that hold a tile's B rows [c0, c0 + ncol).
__host__ __device__ __forceinline__ int n_boxes(int ncol) { return (ncol + BM - 1) / BM; }

// A diagonal tile's A rows [r0, r0 + BM) are one of the 128-row boxes of its
// B rows: the tile loads B only and reads A from B's box diag_box (-1: not a
// diagonal tile).
__host__ __device__ __forceinline__ int diag_box(int r0, int c0, int ncol) {
    const int d = r0 - c0;
    return d >= 0 && d % BM == 0 && d < n_boxes(ncol) * BM ? d / BM : -1;
}

// Entry (a, b) of V (antenna-feed indices in the cover's order) from the 2 x 2
// block g of G, written to its redundant group's slot if it computes one.
__device__ __forceinline__ void put_unique(const HerkOut& ho, float2* Vb, int a, int b, float g00, float g01,
                                           float g10, float g11, float unscale) {
    const int nf = ho.n_feed;
    const int aa = a / nf, pa = a - aa * nf, bb = b / nf, pb = b - bb * nf;
    const int e = ho.uidx[aa * ho.n_ant + bb];
    if (e < 0) return;
    const int grp = e >> 1;
    const bool cj = (e & 1) != 0;
    const float re = ((g00 + g11) * unscale) * unscale;
    const float im = a == b ? 0.f : ((g10 - g01) * unscale) * unscale;
    Vb[((long long)grp * nf + (cj ? pb : pa)) * nf + (cj ? pa : pb)] = make_float2(re, cj ? -im : im);
}

template <int BN>
__device__ __forceinline__ Unit decode_unit(int u, int n_tiles, int S, const int* __restrict__ order,
                                            const Inst* __restrict__ inst, int inst0, const LiveTables& lt,
                                            int n_ax, int rows, const HerkOut& ho) {
    Unit w;
    const int tile = u % n_tiles;
    const int rest = u / n_tiles;
    const int ks = rest % S;
    w.slot = order[rest / S];
    w.part = (w.slot * n_tiles + tile) * S + ks;
    if (ho.tl) {
        const TileDesc d = ho.tl[tile];
        w.r0 = d.r0;
        w.c0 = d.c0;
        w.ncol = d.ncol;
        w.rlim = d.rlim;
        w.clim = d.clim;
    } else {
        int ti;
        tile_at<BN>(tile, rows, ti, w.c0, w.ncol);
        w.r0 = ti * BM;
        w.rlim = w.clim = rows;
    }
    const long long K = (long long)lt.n_live[inst[inst0 + w.slot].t] * n_ax;
    const long long KB = ((K + kKPad - 1) / kKPad * kKPad) / bk_for<BN>();
    w.kb0 = (int)(KB * ks / S);
    w.kb1 = (int)(KB * (ks + 1) / S);
    return w;
}

// order[r] = the slot with the r-th largest live count (ties by slot).
__global__ void k_slot_order(const Inst* __restrict__ inst, int inst0, int n_slots, LiveTables lt,
                             int* __restrict__ order) {
    for (int i = threadIdx.x; i < n_slots; i += blockDim.x) {
        const int ki = lt.n_live[inst[inst0 + i].t];
        int rank = 0;
        for (int j = 0; j < n_slots; ++j) {
            const int kj = lt.n_live[inst[inst0 + j].t];
            rank += (kj > ki) || (kj == ki && j < i);
        }
        order[rank] = i;
    }
}

// Persistent HERK.  Warp 0 fetches units dynamically (one atomic counter per
// launch), streams their U blocks with TMA and broadcasts each unit id to the
// MMA warp and the epilogue warps through a shared-memory queue; the ring
// and the two TMEM buffers carry across units, so the MMA warp starts the
// next unit while the epilogue writes out the last one.
//
// With ZP != 0 the kernel also carries Z_WARPS warps that build the U planes
// of the next batch (zj, written to the other workspace set) with the Z-build
// core (precision ZP, ZA axes, ZF feeds) while the tensor cores work on this
// batch: the two use different units (integer/FP32 pipes and HBM writes vs
// the tensor pipe), and nothing in one waits on the other.
template <int BN, int ZP = 0, int ZA = 1, int ZF = 1>
__global__ void __launch_bounds__(Cfg<BN, zwarps(ZP, ZA, ZF)>::THREADS, 1)
k_herk_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
          const Inst* __restrict__ inst, int inst0, LiveTables lt, int n_ax, uint32_t idesc, int fp16,
          const float* __restrict__ amax, float2* __restrict__ V, int N, int n_tiles, int n_units, int S,
          int flush, const int* __restrict__ order, int* __restrict__ counter, float* __restrict__ partial,
          int* __restrict__ err, const __grid_constant__ ZJob zj, const HerkOut ho) {
    constexpr bool FZ = ZP != 0;
    using C = Cfg<BN, zwarps(ZP, ZA, ZF)>;
    constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES, A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES;
    constexpr int BK = C::BK, SUB = C::SUB;
    constexpr int QD = C::QDEPTH;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // barriers: full[STAGES], empty[STAGES], tfull[2], tempty[2], qfull[QD], qempty[QD]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    int* qslot = reinterpret_cast<int*>(bars + 2 * STAGES + 4 + 2 * QD);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(qslot + QD);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* zsw = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 512);  // 16 floats per Z warp

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * STAGES + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * STAGES + 2 + b]); };
    auto qfull = [&](int q) { return smem_u32(&bars[2 * STAGES + 4 + q]); };
    auto qempty = [&](int q) { return smem_u32(&bars[2 * STAGES + 4 + QD + q]); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull(b), 1); mbar_init(tempty(b), C::EPI_WARPS); }
        for (int q = 0; q < QD; ++q) { mbar_init(qfull(q), 1); mbar_init(qempty(q), 1 + C::EPI_WARPS); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;  // k-blocks loaded so far (ring position)
            for (int n = 0;; ++n) {
                int u = atomicAdd(counter, 1);
                if (u >= n_units) u = -1;
                const int q = n % QD;
                if (!wait_bounded(qempty(q), ((uint32_t)(n / QD) & 1u) ^ 1u, abort_flag, err)) break;
                qslot[q] = u;
                mbar_arrive(qfull(q));
                if (u < 0) break;
                const Unit w = decode_unit<BN>(u, n_tiles, S, order, inst, inst0, lt, n_ax, 2 * N, ho);
                const bool diag = diag_box(w.r0, w.c0, w.ncol) >= 0;
                const int nb = BN == 128 ? 1 : n_boxes(w.ncol);  // full tiles at 128 columns
                const uint32_t bytes = (uint32_t)(2 * nb * SUB + (diag ? 0 : 2 * A_BYTES));
                bool ok = true;
                for (int kb = w.kb0; kb < w.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(empty(s), ph ^ 1u, abort_flag, err)) { ok = false; break; }
                    mbar_expect_tx(full(s), bytes);
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    const int x = kb * BK;
                    if (!diag) {
                        tma_load_3d(st, &map_hi, x, w.r0, w.slot, full(s));
                        tma_load_3d(st + A_BYTES, &map_lo, x, w.r0, w.slot, full(s));
                    }
                    for (int h = 0; h < nb; ++h) {
                        tma_load_3d(st + 2 * A_BYTES + h * SUB, &map_hi, x, w.c0 + h * BM, w.slot, full(s));
                        tma_load_3d(st + 2 * A_BYTES + B_BYTES + h * SUB, &map_lo, x, w.c0 + h * BM, w.slot, full(s));
                    }
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, cg = 0;  // ring position, TMEM chunks issued so far
            for (int n = 0;; ++n) {
                const int q = n % QD;
                if (!wait_bounded(qfull(q), (uint32_t)(n / QD) & 1u, abort_flag, err)) break;
                const int u = qslot[q];
                mbar_arrive(qempty(q));
                if (u < 0) break;
                const Unit w = decode_unit<BN>(u, n_tiles, S, order, inst, inst0, lt, n_ax, 2 * N, ho);
                // A's offset in the stage: its own slot, or the matching half of B
                const int dh = diag_box(w.r0, w.c0, w.ncol);
                const uint32_t a_off = dh < 0 ? 0u : (uint32_t)(2 * A_BYTES + dh * SUB);
                const uint32_t a_lo_off = dh < 0 ? (uint32_t)A_BYTES : a_off + (uint32_t)B_BYTES;
                // N of the tile's MMAs: its width
                const uint32_t id = BN == 128 ? idesc : (idesc & ~(0x3Fu << 17)) | ((uint32_t)(w.ncol >> 3) << 17);
                bool ok = true;
                for (int kc = w.kb0; kc < w.kb1 && ok; kc += flush, ++cg) {
                    const int buf = C::SB ? 0 : cg & 1;
                    const uint32_t ph = C::SB ? (uint32_t)cg & 1u : (uint32_t)(cg >> 1) & 1u;
                    if (!wait_bounded(tempty(buf), ph ^ 1u, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                    const int kc_end = min(w.kb1, kc + flush);
                    uint32_t acc = 0;
                    for (int kb = kc; kb < kc_end; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t sph = (uint32_t)(it / STAGES) & 1u;
                        if (!wait_bounded(full(s), sph, abort_flag, err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t st = sbase + s * STAGE_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t a_hi = sdesc_k<BK>(st + a_off + kk * 32);
                            const uint64_t a_lo = sdesc_k<BK>(st + a_lo_off + kk * 32);
                            const uint64_t b_hi = sdesc_k<BK>(st + 2 * A_BYTES + kk * 32);
                            const uint64_t b_lo = sdesc_k<BK>(st + 2 * A_BYTES + B_BYTES + kk * 32);
                            tc_mma(d, a_hi, b_hi, id, acc);
                            acc = 1;
                            tc_mma(d, a_hi, b_lo, id, 1);
                            tc_mma(d, a_lo, b_hi, id, 1);
                        }
                        tc_commit(empty(s));
                    }
                    tc_commit(tfull(buf));
                }
                if (!ok) break;
            }
        }
    } else if (!FZ || warp < 2 + C::EPI_WARPS) {
        // epilogue warps: TMEM lane quadrant q4, 128-column group h
        const int ew = warp - 2;
        const int q4 = warp & 3, h = ew >> 2;
        int cg = 0;
        for (int n = 0;; ++n) {
            const int qi = n % QD;
            if (!wait_bounded(qfull(qi), (uint32_t)(n / QD) & 1u, abort_flag, err)) break;
            const int u = qslot[qi];
            __syncwarp();
            if (lane == 0) mbar_arrive(qempty(qi));
            if (u < 0) break;
            const Unit w = decode_unit<BN>(u, n_tiles, S, order, inst, inst0, lt, n_ax, 2 * N, ho);
            const int rl = q4 * 32 + lane;  // row of the tile held by this thread
            const int r = w.r0 + rl;
            const int a = r >> 1;
            const bool even = (lane & 1) == 0;
            float2* Vb = V + inst[inst0 + w.slot].v_off;
            const int c0 = w.c0 + h * 128;
            // columns of this warp's 128 inside the tile (all of them at 128 columns)
            const int ncv = BN == 128 ? 128 : w.ncol - h * 128;
            // undo the FP16 scaling 2^e of both operands: two exact power-of-two steps
            const float unscale = fp16 ? ldexpf(1.f, -fp16_scale_exp(amax[w.slot])) : 1.f;
            // one 32-column chunk of the tile (columns c0 + 32 g ...): raw partial
            // tile, or the 2 x 2 blocks of G folded into V
            auto write_chunk = [&](auto ncol, int g, const float* x) {
                constexpr int NCOL = decltype(ncol)::value;
                if (S > 1) {
                    // column-major [BN][128] (coalesced along rows)
                    float* p = partial + (long long)w.part * (BN * BM) + (long long)(h * 128 + g * NCOL) * BM + rl;
#pragma unroll
                    for (int j = 0; j < NCOL; ++j) p[j * BM] = x[j];
                    return;
                }
#pragma unroll
                for (int jj = 0; jj < NCOL / 2; ++jj) {
                    const float x0 = x[2 * jj], x1 = x[2 * jj + 1];
                    const float y0 = __shfl_xor_sync(0xffffffffu, x0, 1);
                    const float y1 = __shfl_xor_sync(0xffffffffu, x1, 1);
                    const float g00 = even ? x0 : y0, g01 = even ? x1 : y1;
                    const float g10 = even ? y0 : x0, g11 = even ? y1 : x1;
                    const int b = (c0 + g * NCOL + 2 * jj) >> 1;
                    if (ho.uidx) {  // one value per redundant group
                        if ((jj & 1) == (lane & 1) && r < w.rlim && 2 * b < w.clim && a < N && b < N)
                            put_unique(ho, Vb, a, b, g00, g01, g10, g11, unscale);
                        continue;
                    }
                    if ((jj & 1) == (lane & 1) && a < N && b < N && a >= b) {
                        const float re = ((g00 + g11) * unscale) * unscale;
                        // autocorrelations are real: the tensor core rounds the two
                        // symmetric entries of G separately, so drop that residue
                        const float im = a == b ? 0.f : ((g10 - g01) * unscale) * unscale;
                        Vb[(long long)a * N + b] = make_float2(re, im);
                        if (a != b) Vb[(long long)b * N + a] = make_float2(re, -im);
                    }
                }
            };
            bool ok = true;
            if constexpr (!FZ) {
                // running sums in registers
                float run[128];
#pragma unroll
                for (int i = 0; i < 128; ++i) run[i] = 0.f;
                for (int kc = w.kb0; kc < w.kb1; kc += flush, ++cg) {
                    const int buf = cg & 1;
                    const uint32_t ph = (uint32_t)(cg >> 1) & 1u;
                    if (!wait_bounded(tfull(buf), ph, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ta = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * BN + h * 128);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (g * 32 >= ncv) break;
                        uint32_t rr[32];
                        tmem_ld32(ta + g * 32, rr);
                        tmem_wait_ld(rr);
#pragma unroll
                        for (int i = 0; i < 32; ++i) run[g * 32 + i] += __uint_as_float(rr[i]);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty(buf));
                }
                if (!ok || *abort_flag) break;
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    if (g * 32 < ncv) write_chunk(std::integral_constant<int, 32>{}, g, run + g * 32);
            } else {
                // running sums in TMEM columns [RUN, RUN + BN) of this warp's lanes
                // and 128-column group, 16 columns at a time
                const uint32_t tl = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(h * 128);
                const uint32_t trun = tl + C::RUN;
                bool any = false;
                for (int kc = w.kb0; kc < w.kb1; kc += flush, ++cg) {
                    const int buf = C::SB ? 0 : cg & 1;
                    const uint32_t ph = C::SB ? (uint32_t)cg & 1u : (uint32_t)(cg >> 1) & 1u;
                    if (!wait_bounded(tfull(buf), ph, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ta = tl + (uint32_t)(buf * BN);
#pragma unroll 1
                    for (int g = 0; g < 8 && g * 16 < ncv; ++g) {
                        uint32_t acc[16];
                        tmem_ld16(ta + g * 16, acc);
                        tmem_wait_ld16(acc);
                        if (any) {
                            uint32_t sum[16];
                            tmem_ld16(trun + g * 16, sum);
                            tmem_wait_ld16(sum);
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                acc[i] = __float_as_uint(__uint_as_float(sum[i]) + __uint_as_float(acc[i]));
                        }
                        tmem_st16(trun + g * 16, acc);
                    }
                    tmem_wait_st();
                    any = true;
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty(buf));
                }
                if (!ok || *abort_flag) break;
#pragma unroll 1
                for (int g = 0; g < 8 && g * 16 < ncv; ++g) {
                    float x[16];
                    if (any) {
                        uint32_t sum[16];
                        tmem_ld16(trun + g * 16, sum);
                        tmem_wait_ld16(sum);
#pragma unroll
                        for (int i = 0; i < 16; ++i) x[i] = __uint_as_float(sum[i]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) x[i] = 0.f;
                    }
                    write_chunk(std::integral_constant<int, 16>{}, g, x);
                }
            }
        }
    } else if constexpr (FZ) {
        // Z build of the next batch
        if (zj.n_groups > 0) {
            const int zw = warp - 2 - C::EPI_WARPS;
            zcore::zjob_warp<ZP, ZA, ZF>(zj, blockIdx.x * C::Z_WARPS + zw, gridDim.x * C::Z_WARPS, zsw + zw * 16);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS));
    }
}

// Sum the S partial tiles of every (slot, tile) in a fixed order and fold the
// 2 x 2 blocks of G into V (lower triangle + conjugate mirror).
template <int BN>
__global__ void __launch_bounds__(256)
k_herk_finalize(const Inst* __restrict__ inst, int inst0, int fp16, const float* __restrict__ amax,
                const float* __restrict__ partial, float2* __restrict__ V, int N, int n_tiles, int S,
                const HerkOut ho) {
    const int st = blockIdx.x;
    const int slot = st / n_tiles, tile = st % n_tiles;
    int r0, c0, ncol, rlim = 2 * N, clim = 2 * N;
    if (ho.tl) {
        const TileDesc d = ho.tl[tile];
        r0 = d.r0;
        c0 = d.c0;
        ncol = d.ncol;
        rlim = d.rlim;
        clim = d.clim;
    } else {
        int ti;
        tile_at<BN>(tile, 2 * N, ti, c0, ncol);
        r0 = ti * BM;
    }
    const int q = blockIdx.y * 256 + threadIdx.x;  // 2 x 2 block index within the tile
    const int rp = q % (BM / 2), cp = q / (BM / 2);
    const int r = 2 * rp, c = 2 * cp;
    const int a = (r0 + r) >> 1, b = (c0 + c) >> 1;
    if (c >= ncol || a >= N || b >= N || r0 + r >= rlim || c0 + c >= clim) return;
    if (!ho.uidx && a < b) return;
    float g00 = 0.f, g10 = 0.f, g01 = 0.f, g11 = 0.f;
    for (int ks = 0; ks < S; ++ks) {
        const float* p = partial + ((long long)st * S + ks) * (BN * BM);
        const float2 v0 = *reinterpret_cast<const float2*>(p + (long long)c * BM + r);
        const float2 v1 = *reinterpret_cast<const float2*>(p + (long long)(c + 1) * BM + r);
        g00 += v0.x;
        g10 += v0.y;
        g01 += v1.x;
        g11 += v1.y;
    }
    const float unscale = fp16 ? ldexpf(1.f, -fp16_scale_exp(amax[slot])) : 1.f;
    float2* Vb = V + inst[inst0 + slot].v_off;
    if (ho.uidx) {
        put_unique(ho, Vb, a, b, g00, g01, g10, g11, unscale);
        return;
    }
    const float re = ((g00 + g11) * unscale) * unscale;
    const float im = a == b ? 0.f : ((g10 - g01) * unscale) * unscale;
    Vb[(long long)a * N + b] = make_float2(re, im);
    if (a != b) Vb[(long long)b * N + a] = make_float2(re, -im);
}

bool make_map(CUtensorMap* map, const void* base, long long k_pitch, int rows, int n_slots, bool fp16, int bk) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)k_pitch, (cuuint64_t)rows, (cuuint64_t)n_slots};
    cuuint64_t strides[2] = {(cuuint64_t)k_pitch * 2, (cuuint64_t)k_pitch * 2 * rows};
    cuuint32_t box[3] = {(cuuint32_t)bk, BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int ZP = 0, int ZA = 1, int ZF = 1>
cudaError_t launch_bn(const CUtensorMap& mh, const CUtensorMap& ml, const Inst* d_inst, int inst0, int n_inst,
                      LiveTables lt, int n_ax, int fp16, const float* d_amax, float2* d_v, int N, int rows,
                      int flush, int split, int n_ctas, int* d_sched, float* d_partial, int* d_err,
                      const ZJob* zj, const HerkOut& ho, cudaStream_t st, long long* launches) {
    using C = Cfg<BN, zwarps(ZP, ZA, ZF)>;
    flush *= 64 / C::BK;  // the option counts 64-source blocks
    const int n_tiles = ho.tl ? ho.n_tl : n_tiles_for<BN>(rows);
    const int n_units = n_tiles * n_inst * split;
    int* order = d_sched;            // [n_inst]
    int* counter = d_sched + n_inst;  // one int
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_slot_order<<<1, 256, 0, st>>>(d_inst, inst0, n_inst, lt, order);
    // with a fused Z build every SM takes part (CTAs without HERK units build Z)
    const int grid = ZP != 0 ? std::max(1, n_ctas) : std::max(1, std::min(n_ctas, n_units));
    ZJob z{};
    if (zj) z = *zj;
    k_herk_tc<BN, ZP, ZA, ZF><<<grid, C::THREADS, C::SMEM, st>>>(mh, ml, d_inst, inst0, lt, n_ax,
                                                                 idesc_for(fp16 != 0, BN), fp16, d_amax, d_v, N,
                                                                 n_tiles, n_units, split, flush, order, counter,
                                                                 d_partial, d_err, z, ho);
    *launches += 2;
    if (split > 1) {
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 g2(n_tiles * n_inst, (BM / 2) * (BN / 2) / 256);
        k_herk_finalize<BN><<<g2, 256, 0, st>>>(d_inst, inst0, fp16, d_amax, d_partial, d_v, N, n_tiles, split, ho);
        *launches += 1;
    }
    return cudaGetLastError();
}

// A bounded mbarrier wait that nothing completes: one thread waits limit_ns
// through the same wait as every tensor-core kernel, then records the device
// timeout in err and returns (the failure path of those kernels, without a
// fault).
__global__ void k_wait_probe(int* __restrict__ err, unsigned long long limit_ns) {
    __shared__ alignas(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) wait_bounded(smem_u32(&bar), 0u, &abort_flag, err, limit_ns);
}

}  // namespace

cudaError_t launch_wait_probe(int* d_err, double limit_s, cudaStream_t st) {
    if (!d_err || !(limit_s > 0) || limit_s > 10) return cudaErrorInvalidValue;
    k_wait_probe<<<1, 32, 0, st>>>(d_err, (unsigned long long)(limit_s * 1e9));
    return cudaGetLastError();
}

bool herk_tc_available() { return get_encode() != nullptr; }

cudaError_t herk_tc_init() {
    const int f1 = Cfg<128, zwarps(2, 1, 1)>::SMEM, f2 = Cfg<128, zwarps(2, 2, 2)>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_herk_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<128>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_herk_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<256>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_herk_tc<128, 2, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, f1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_herk_tc<128, 2, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, f2);
    const int w1 = Cfg<256, zwarps(2, 1, 1)>::SMEM, w2 = Cfg<256, zwarps(2, 2, 2)>::SMEM;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_herk_tc<256, 2, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, w1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_herk_tc<256, 2, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, w2);
    return e;
}

bool herk_tc_fusable(int bn, int zprec, int n_ax, int n_feed) {
    return (bn == 128 || bn == 256) && zprec == 2 && n_ax == n_feed && (n_ax == 1 || n_ax == 2);
}

int herk_tc_units(int rows, int n_slots, int split, int bn) {
    return (bn == 128 ? n_tiles_for<128>(rows) : n_tiles_for<256>(rows)) * n_slots * split;
}

cudaError_t launch_herk_tc(const Inst* d_inst, int inst0, int n_inst, LiveTables lt, int n_ax,
                           const __nv_bfloat16* d_hi, const __nv_bfloat16* d_lo, int rows, long long k_pitch,
                           int n_slots, int fp16, const float* d_amax, float2* d_v, int N, int flush, int split,
                           int bn, int n_ctas, int* d_sched, float* d_partial, int* d_err, const ZJob* zj,
                           int zprec, const HerkOut* out, cudaStream_t st, long long* launches) {
    CUtensorMap mh, ml;
    const int bk = bn == 128 ? bk_for<128>() : bk_for<256>();
    if (!make_map(&mh, d_hi, k_pitch, rows, n_slots, fp16, bk) || !make_map(&ml, d_lo, k_pitch, rows, n_slots, fp16, bk))
        return cudaErrorInvalidValue;
    if (flush < 1) flush = 4;
    if (split < 1) split = 1;
    if ((split > 1 && !d_partial) || !d_sched || n_inst > 4096) return cudaErrorInvalidValue;
    HerkOut ho{};
    if (out) {
        ho = *out;
        // a listed cover at 128 columns holds full-width tiles only
        if (ho.n_feed < 1 || ho.n_ant < 1 || !ho.uidx || (ho.tl && ho.n_tl < 1)) return cudaErrorInvalidValue;
    }
#define MV_LB(BN_, ZP_, ZA_, ZF_)                                                                                \
    return launch_bn<BN_, ZP_, ZA_, ZF_>(mh, ml, d_inst, inst0, n_inst, lt, n_ax, fp16, d_amax, d_v, N, rows, flush, \
                                         split, n_ctas, d_sched, d_partial, d_err, zj, ho, st, launches)
    if (zj) {
        if (!herk_tc_fusable(bn, zprec, zj->m.n_ax, zj->m.n_feed)) return cudaErrorInvalidValue;
        if (bn == 256) {
            if (zj->m.n_ax == 1) MV_LB(256, 2, 1, 1);
            MV_LB(256, 2, 2, 2);
        }
        if (zj->m.n_ax == 1) MV_LB(128, 2, 1, 1);
        MV_LB(128, 2, 2, 2);
    }
    if (bn == 128) MV_LB(128, 0, 1, 1);
    MV_LB(256, 0, 1, 1);
#undef MV_LB
}

}  // namespace mv
