// mlp_tc.cu -- the learned beam's forward pass on the sm_103a tensor cores,
// fused with the beam-times-flux step of the simulator: for every row
// (antenna beam b, live source s) of one instance it evaluates the network
// and writes WA[b][comp][s] = sqrt(I_s(nu)) A^{pk}_b(s) (or, for a polarised
// sky, A M with the coherency square root, eq. "fullz") -- Algorithm 2 step
// (ii) of arXiv:2312.09763 with the network in place of the interpolation of
// Sec. 2.4.
//
// The network (mlp.cu): x = (az / 2 pi, za / (pi/2), (nu - nu_mid) / nu_half),
// f = [sin(2 pi B x), cos(2 pi B x), e_b, 0...] (d0p columns), h_l = relu(W_l
// h_{l-1} + b_l) for the hidden layers, y = W_out h + b_out.  Operands are
// BF16, accumulation FP32 in TMEM, as in the training kernels.
//
// The first layer is linear in its input, and of its input only the
// embedding e_b depends on the beam: W_0 f + b_0 = P_s + C_b with P_s the
// product of W_0's Fourier columns with the source's features (the same for
// every beam) and C_b = W_0's embedding columns times e_b, plus b_0.  So P is
// computed once per live source of the instance (k_src_first, FP32 on the
// CUDA cores from the same BF16 features and weights) and C once per beam
// (k_beam_first), and the fused kernel starts every row at h_1 = relu(P_s +
// C_b): the Fourier features and the first layer's products are not
// repeated for each of the n_beam beams.
//
// One persistent CTA per SM walks 256-row tiles of 8 beams x 32 consecutive
// live sources (one beam per 32 rows), held as two 128-row sub-tiles with
// their own activation panels, TMEM accumulators (columns 0 and 256) and
// barriers.  The sub-tiles take turns on the tensor pipe: warp 1 (which owns
// TMEM) issues one sub-tile's layer (M = 128, N = H, K = 16) while the other
// sub-tile's 8 epilogue warps drain its previous layer through bias and ReLU
// back into its shared-memory activation panels, so the tensor pipe does not
// wait for an epilogue.  Warp 0 streams each layer's weight panels (64 input
// columns x H rows, 128-byte swizzle, kept in L2) with TMA through a ring of
// two slots, once per sub-tile.  A sub-tile's 8 warps (one per TMEM lane
// quadrant and half of the columns) also write its h_1 -- split by 16-column
// groups, each lane loading its source's P values once for the sub-tile's 4
// beams and the beams' C from shared memory, where it was staged a tile
// ahead -- and, after the output layer, its WA: 32 consecutive sources of one
// beam per warp, with streaming stores.  Every mbarrier wait is bounded
// (tc.cuh).
#include <cuda_bf16.h>

#include <algorithm>
#include "common.cuh"
#include "tc.cuh"

namespace mv {
namespace {

using namespace tc;

constexpr int TM = 128;          // rows per sub-tile (one TMEM accumulator)
constexpr int TILE = 2 * TM;     // rows per tile: two sub-tiles
constexpr int KP = 64;           // input columns per swizzled panel (128 B of BF16)
constexpr int MAXL = 8;          // hidden layers at most
constexpr int A_PANEL = TM * 128;                // 16 KB
constexpr int W_PANEL_MAX = 256 * 128;           // 32 KB (H = 256)
constexpr int O_PANEL = 16 * 128;                // 2 KB (output rows padded to 16 with zeros)
constexpr int SUB_A = 4 * A_PANEL;               // 64 KB of activations per sub-tile
constexpr int SMEM_A = 2 * SUB_A;                // 128 KB
constexpr int NSLOT = 2;                         // weight-panel ring
constexpr int TMEM_COLS = 512;                   // two 256-column accumulators
constexpr int SMEM_W = NSLOT * W_PANEL_MAX;      // 64 KB
constexpr int SMEM_O = 4 * O_PANEL;              // 8 KB
constexpr int SMEM_BIAS = (MAXL + 1) * 256 * 4;  // every layer's biases
constexpr int MAXF = 128;                         // Fourier frequencies at most
constexpr int NEPI = 16;                          // epilogue warps: four per TMEM lane quadrant
// per-row values gathered ahead of use with cp.async for the WA writers:
// (m00, Re m10, Im m10, m11) or (flux, 0, 0, 0), and the spectral index
constexpr int SMEM_GATHER = TILE * 16 + TILE * 4;
constexpr int SMEM_C = 8 * 256 * 4;               // C rows of the next tile's 8 beams
constexpr int SMEM_BYTES = SMEM_A + SMEM_W + SMEM_O + SMEM_BIAS + SMEM_GATHER + SMEM_C + 256 + 1024;
constexpr int THREADS = (2 + NEPI) * 32;
// P: sources in blocks of 32, each block [H / 4][32][4] floats, so that the
// 32 consecutive rows of a warp read 512 contiguous bytes per float4 column
// group
constexpr int SRC_BLK = 32;

struct Maps {
    CUtensorMap w[MAXL + 1];  // hidden layers, then the output layer
};

struct Net {
    int H, depth, n_beam, n_out;
    const float* p;  // FP32 parameters (biases)
    long long off_b[MAXL + 1];
    const float* P;  // first-layer products of the Fourier features, per live source (SRC_BLK layout)
    const float* C;  // first-layer embedding products plus b_0, per beam: [n_beam][H]
};

// Shared-memory address of the 16-byte chunk holding input columns
// [8 j, 8 j + 8) of panel `panel`, row r (128-byte swizzle: chunk j ^ (r & 7)).
__device__ __forceinline__ uint32_t a_chunk(uint32_t a_base, int r, int col) {
    const int panel = col / KP, j = (col % KP) / 8;
    return a_base + panel * A_PANEL + r * 128 + ((j ^ (r & 7)) << 4);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// max(lo, 0) in the low half, max(hi, 0) in the high half, rounded to BF16.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Ampere-style asynchronous global -> shared copies of 4, 8 or 16 bytes.
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t saddr, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr), "l"(g), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }



__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16(x)); }

// ------------------------------------------------- per-source first layer
// P_s = sum over the 2F Fourier columns c of W_0[j][c] f_c(s), FP32, for the
// 32 live sources of block blockIdx.x of instance (t, nu); the features are
// the fused pass's own (turns reduced to [-1/2, 1/2], fast sine and cosine,
// rounded to BF16), the weights W_0's BF16 copy.  Rows past K are zeros.
// Dynamic shared memory: features [2F][32] and the block's P [32][H + 4].
struct SrcArgs {
    int F, H, d0p;
    float nu_mid, nu_half;
    const float* Bf;               // [F][3]
    const __nv_bfloat16* w0;       // W_0, [H][d0p]
};

__global__ void __launch_bounds__(256)
k_src_first(SrcArgs a, LiveTables lt, int t, int K, float nu, float* __restrict__ P) {
    extern __shared__ float sm[];
    const int F = a.F, H = a.H, F2 = 2 * a.F, ldp = H + 4;
    float* fs = sm;             // [2F][32]
    float* ps = sm + F2 * 32;   // [32][H + 4]
    const int s0 = blockIdx.x * SRC_BLK;
    const float x2 = (nu - a.nu_mid) / a.nu_half;
    for (int q = threadIdx.x; q < F * SRC_BLK; q += blockDim.x) {
        const int f = q / SRC_BLK, i = q % SRC_BLK, s = s0 + i;
        float sv = 0.f, cv = 0.f;
        if (s < K) {
            const float2 azza = lt.azza[(long long)t * lt.pitch + s];
            const float x0 = azza.x * 0.15915494309189535f;  // az / 2 pi
            const float x1 = azza.y * 0.63661977236758134f;  // za / (pi / 2)
            float ph = a.Bf[3 * f] * x0 + a.Bf[3 * f + 1] * x1 + a.Bf[3 * f + 2] * x2;
            ph -= rintf(ph);
            __sincosf(6.283185307179586f * ph, &sv, &cv);
        }
        fs[f * SRC_BLK + i] = bf16_round(sv);
        fs[(F + f) * SRC_BLK + i] = bf16_round(cv);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        float acc[SRC_BLK];
#pragma unroll
        for (int i = 0; i < SRC_BLK; ++i) acc[i] = 0.f;
        const __nv_bfloat16* wr = a.w0 + (long long)j * a.d0p;
        for (int c8 = 0; c8 < F2; c8 += 8) {
            const uint4 wv = *reinterpret_cast<const uint4*>(wr + c8);  // rows of d0p % 16 == 0 elements
            const uint32_t wp[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t pr = wp[k >> 1];
                const float w = __uint_as_float((k & 1) ? (pr & 0xFFFF0000u) : (pr << 16));
                const float4* f4 = reinterpret_cast<const float4*>(fs + (c8 + k) * SRC_BLK);
#pragma unroll
                for (int i4 = 0; i4 < SRC_BLK / 4; ++i4) {
                    const float4 v = f4[i4];
                    acc[4 * i4] = fmaf(w, v.x, acc[4 * i4]);
                    acc[4 * i4 + 1] = fmaf(w, v.y, acc[4 * i4 + 1]);
                    acc[4 * i4 + 2] = fmaf(w, v.z, acc[4 * i4 + 2]);
                    acc[4 * i4 + 3] = fmaf(w, v.w, acc[4 * i4 + 3]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < SRC_BLK; ++i) ps[i * ldp + j] = acc[i];
    }
    __syncthreads();
    // the block's [H / 4][32][4] floats, contiguous in P
    float4* dst = reinterpret_cast<float4*>(P + (long long)blockIdx.x * SRC_BLK * H);
    for (int q = threadIdx.x; q < SRC_BLK * H / 4; q += blockDim.x) {
        const int g = q / SRC_BLK, i = q % SRC_BLK;
        dst[q] = *reinterpret_cast<const float4*>(ps + i * ldp + 4 * g);
    }
}

// C_b = b_0 + W_0's embedding columns times e_b (rounded to BF16 as in the
// features), FP32; one block per beam, one thread per output.
__global__ void k_beam_first(SrcArgs a, int E, const float* __restrict__ p, long long off_b0, long long off_emb,
                             float* __restrict__ C) {
    const int b = blockIdx.x;
    for (int j = threadIdx.x; j < a.H; j += blockDim.x) {
        float acc = p[off_b0 + j];
        const __nv_bfloat16* wr = a.w0 + (long long)j * a.d0p + 2 * a.F;
        for (int e = 0; e < E; ++e) acc = fmaf(__bfloat162float(wr[e]), bf16_round(p[off_emb + (long long)b * E + e]), acc);
        C[(long long)b * a.H + j] = acc;
    }
}

// ------------------------------------------------------------ fused pass
// h_1 = relu(P_s + C_b) of a tile (beams b0 .. b0 + 7, sources s0 .. s0 +
// 31) into the activation panels, zeros for rows past the instance.  The
// rows need no TMEM, so the work is split by columns: epilogue warp ew takes
// the 16 columns [16 g, 16 g + 16) with g = ew mod (H / 16) and every
// (16 / (H / 16))-th beam from ew / (H / 16) on; lane = source.  Each lane
// loads its source's 16 values of P once (a warp reads 512 contiguous bytes
// per float4 column group, and the tile's P block is read once) and adds the
// beams' C values, which are the same for every lane (broadcast loads).
// Each sub-tile's 8 epilogue warps write its h_1 (4 beams x 32 sources):
// warp w (0..7) takes the 16-column groups g = w, w + 8, ... below H / 16,
// for the sub-tile's 4 beams.  first_stage copies the warp's slices of the
// beams' C rows into shared memory a tile ahead (cp.async, 16 bytes per
// lane); first_store loads the sources' P values per group (a warp reads 512
// contiguous bytes per float4 column group) and writes the panels.
// cs: C rows of the tile's 8 beams in shared memory, [8][256] floats.
__device__ __forceinline__ void first_stage(int w, int u, int lane, int H, int b0, int n_beam,
                                            const float* __restrict__ C, float* cs) {
    const int g = w + 8 * (lane >> 4), jj = (lane >> 2) & 3, c = 16 * g + 4 * (lane & 3);
    const int j = 4 * u + jj;
    if (16 * g < H && b0 + j < n_beam)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(cs + j * 256 + c)),
                     "l"(C + (long long)(b0 + j) * H + c)
                     : "memory");
}
__device__ __forceinline__ void first_store(int w, int u, uint32_t ab, int lane, int H, int b0, int n_beam, int s0,
                                            int K, const float* __restrict__ P, const float* cs) {
    const bool svalid = s0 + lane < K;
    const float* pr = P + ((long long)(s0 / SRC_BLK) * H * SRC_BLK + lane * 4);
    for (int g = w; 16 * g < H; g += 8) {
        const int c0 = 16 * g;
        float4 pv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            pv[i] = svalid ? __ldg(reinterpret_cast<const float4*>(pr + (long long)(c0 / 4 + i) * (SRC_BLK * 4)))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * u + jj;
            const bool valid = svalid && b0 + j < n_beam;
            const float4* cr = reinterpret_cast<const float4*>(cs + j * 256 + c0);
            const int r = jj * 32 + lane;  // row of the sub-tile
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8) {
                const float4 p0 = pv[2 * h8], p1 = pv[2 * h8 + 1];
                const float4 k0 = valid ? cr[2 * h8] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 k1 = valid ? cr[2 * h8 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t w0 = relu_bf16x2(p0.x + k0.x, p0.y + k0.y), w1 = relu_bf16x2(p0.z + k0.z, p0.w + k0.w);
                uint32_t w2 = relu_bf16x2(p1.x + k1.x, p1.y + k1.y), w3 = relu_bf16x2(p1.z + k1.z, p1.w + k1.w);
                if (!valid) w0 = w1 = w2 = w3 = 0u;
                st_shared_v4(a_chunk(ab, r, c0 + 8 * h8), w0, w1, w2, w3);
            }
        }
    }
}

// 32 accumulator columns [c0, c0 + 32) of row r through bias and ReLU into
// the activation panels.
__device__ __forceinline__ void drain32(uint32_t ab, int r, int c0, const uint32_t (&x)[32],
                                        const float* __restrict__ bias) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 b0 = *reinterpret_cast<const float4*>(bias + c0 + 8 * j);
        const float4 b1 = *reinterpret_cast<const float4*>(bias + c0 + 8 * j + 4);
        st_shared_v4(a_chunk(ab, r, c0 + 8 * j),
                     relu_bf16x2(__uint_as_float(x[8 * j]) + b0.x, __uint_as_float(x[8 * j + 1]) + b0.y),
                     relu_bf16x2(__uint_as_float(x[8 * j + 2]) + b0.z, __uint_as_float(x[8 * j + 3]) + b0.w),
                     relu_bf16x2(__uint_as_float(x[8 * j + 4]) + b1.x, __uint_as_float(x[8 * j + 5]) + b1.y),
                     relu_bf16x2(__uint_as_float(x[8 * j + 6]) + b1.z, __uint_as_float(x[8 * j + 7]) + b1.w));
    }
}

// Columns [c_beg, c_beg + n) (n a multiple of 32) of a hidden layer's
// accumulator row (TMEM address trow) into the activation panels.
__device__ __forceinline__ void drain_layer(uint32_t trow, uint32_t ab, int r, int c_beg, int n,
                                            const float* __restrict__ bias) {
    for (int c0 = c_beg; c0 < c_beg + n; c0 += 32) {
        uint32_t x[32];
        tmem_ld32(trow + c0, x);
        tmem_wait_ld(x);
        drain32(ab, r, c0, x, bias);
    }
}

__global__ void __launch_bounds__(THREADS, 1)
k_mlp_wa(const __grid_constant__ Maps maps, const __grid_constant__ Net net, Model m, LiveTables lt, int t, int K,
         float ln_ratio, float2* __restrict__ wa, long long wa_pitch, float* __restrict__ amax,
         int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t a_base = smem_u32(smem);
    const uint32_t w_base = a_base + SMEM_A;
    const uint32_t o_base = w_base + SMEM_W;
    float* sbias = reinterpret_cast<float*>(smem + SMEM_A + SMEM_W + SMEM_O);  // [layer][256]
    uint8_t* sgather = smem + SMEM_A + SMEM_W + SMEM_O + SMEM_BIAS;
    float4* g_m = reinterpret_cast<float4*>(sgather);                     // [row of the tile]
    float* g_alpha = reinterpret_cast<float*>(sgather + TILE * 16);       // [row of the tile]
    float* c_rows = reinterpret_cast<float*>(sgather + SMEM_GATHER);     // [beam of the tile][256]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sgather + SMEM_GATHER + SMEM_C);
    // wfull[NSLOT], wfree[NSLOT], afull[2], dfull[2], ofull (afull / dfull per sub-tile)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSLOT + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    auto wfull = [&](int i) { return smem_u32(&bars[i]); };
    auto wfree = [&](int i) { return smem_u32(&bars[NSLOT + i]); };
    auto afull = [&](int u) { return smem_u32(&bars[2 * NSLOT + u]); };
    auto dfull = [&](int u) { return smem_u32(&bars[2 * NSLOT + 2 + u]); };
    const uint32_t ofull = smem_u32(&bars[2 * NSLOT + 4]);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = net.H, D = net.depth;
    // tiles of 8 beams x 32 sources: tile = source block x beam groups + beam group
    const int n_bg = (net.n_beam + 7) / 8;
    const int n_tiles = (K + SRC_BLK - 1) / SRC_BLK * n_bg;
    const int w_panel = H * 128;
    const int np = H / KP;  // input panels of layers 1 .. D (the output layer included)

    // output-layer panels: rows 8..15 stay zero (the tensor map fills rows 0..7)
    for (int i = threadIdx.x; i < SMEM_O / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem + SMEM_A + SMEM_W)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int l = 1; l <= D; ++l) {
        const int n = l == D ? 8 : H;
        for (int i = threadIdx.x; i < n; i += blockDim.x) sbias[l * 256 + i] = net.p[net.off_b[l] + i];
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) { mbar_init(wfull(i), 1); mbar_init(wfree(i), 1); }
        for (int u = 0; u < 2; ++u) { mbar_init(afull(u), NEPI / 2); mbar_init(dfull(u), 1); }
        mbar_init(ofull, 1);
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
            // output layer once: its 8 rows (one 1 KB swizzle atom per panel)
            mbar_expect_tx(ofull, (uint32_t)(np * (O_PANEL / 2)));
            for (int pnl = 0; pnl < np; ++pnl) tma_load_2d(o_base + pnl * O_PANEL, &maps.w[D], pnl * KP, 0, ofull);
            // the hidden layers' panels, once for each sub-tile (in the MMA
            // warp's order), kept in L2 (evict-last) under the stream of WA
            // stores
            const uint64_t pol = policy_evict_last();
            int it = 0;  // weight panels streamed so far (ring position)
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
                for (int l = 1; l < D && ok; ++l)
                    for (int u = 0; u < 2 && ok; ++u)
                        for (int pnl = 0; pnl < np; ++pnl, ++it) {
                            const int sl = it % NSLOT;
                            if (!wait_bounded_spin(wfree(sl), ((uint32_t)(it / NSLOT) & 1u) ^ 1u, abort_flag, err)) { ok = false; break; }
                            mbar_expect_tx(wfull(sl), (uint32_t)w_panel);
                            tma_load_2d_hint(w_base + sl * W_PANEL_MAX, &maps.w[l], pnl * KP, 0, wfull(sl), pol);
                        }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // layer by layer, sub-tile 0 then sub-tile 1: while one sub-tile's
            // epilogue drains a layer, the other's MMAs run
            const uint32_t id_hidden = idesc_f16(false, TM, H), id_out = idesc_f16(false, TM, 16);
            int it = 0;
            int na0 = 0, na1 = 0;
            bool ok = wait_bounded_spin(ofull, 0u, abort_flag, err);
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int l = 1; l <= D && ok; ++l) {
                    const bool out = l == D;
                    for (int u = 0; u < 2 && ok; ++u) {
                        const int na = u ? na1++ : na0++;
                        if (!wait_bounded_spin(afull(u), (uint32_t)na & 1u, abort_flag, err)) { ok = false; break; }
                        tc_fence_after();
                        for (int pnl = 0; pnl < np; ++pnl) {
                            const int sl = it % NSLOT;
                            if (!out) {
                                if (!wait_bounded_spin(wfull(sl), (uint32_t)(it / NSLOT) & 1u, abort_flag, err)) { ok = false; break; }
                                tc_fence_after();
                            }
                            const uint32_t b0 = out ? o_base + pnl * O_PANEL : w_base + sl * W_PANEL_MAX;
                            for (int kk = 0; kk < KP / 16; ++kk)
                                tc_mma(tmem + (uint32_t)(u * 256), sdesc(a_base + u * SUB_A + pnl * A_PANEL + kk * 32),
                                       sdesc(b0 + kk * 32), out ? id_out : id_hidden, (pnl | kk) != 0 ? 1u : 0u);
                            if (!out) {
                                tc_commit(wfree(sl));
                                ++it;
                            }
                        }
                        if (!ok) break;
                        tc_commit(dfull(u));
                    }
                }
            }
        }
    } else {
        // epilogue warps: lane quadrant q, sub-tile u, column half h; the
        // sub-tile's 8 warps are numbered w = (q, h)
        const int q = warp & 3, u = ((warp - 2) >> 2) & 1, h = (warp - 2) >> 3;
        const int w = ((warp - 2) & 3) + 4 * h;
        const int r_loc = q * 32 + lane;  // row within the sub-tile
        const int row = u * TM + r_loc;   // row within the tile
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(u * 256);
        const uint32_t ab = a_base + u * SUB_A;
        const uint32_t my_afull = afull(u), my_dfull = dfull(u);
        const int half = H / 2, c_beg = h * half;
        const int ncomp = net.n_out / 2;
        int nd = 0;
        bool ok = true;
        // row of the network input in a tile: beam b (one per warp), live
        // source s (one per lane)
        auto row_of = [&](int tile, bool& valid, int& b, int& s) {
            b = (tile % n_bg) * 8 + u * 4 + q;
            s = (tile / n_bg) * SRC_BLK + lane;
            valid = b < net.n_beam && s < K;
            if (!valid) b = s = 0;
        };
        auto stage_tile = [&](int tile) {
            first_stage(w, u, lane, H, (tile % n_bg) * 8, net.n_beam, net.C, c_rows);
            cp_async_commit();
        };
        // h_1 of the sub-tile into its activation panels, then the MMA warp
        // may go (the caller has waited for the tile's staged C rows)
        auto start_tile = [&](int tile) {
            __syncwarp();
            first_store(w, u, ab, lane, H, (tile % n_bg) * 8, net.n_beam, (tile / n_bg) * SRC_BLK, K, net.P, c_rows);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(my_afull);
        };
        // Per tile: the WA writers (half 0) request their source's flux,
        // spectral index (and coherency root) once the sub-tile's first
        // product is done; they land in shared memory while the layers run.
        // After the output layer the warps read its accumulator, write the
        // next tile's h_1 (the MMA warp starts on it), and then scale and
        // store this tile's WA.
        int tile = blockIdx.x;
        if (tile < n_tiles) {
            stage_tile(tile);
            cp_async_wait_all();
            start_tile(tile);
        }
        for (; tile < n_tiles && ok; tile += gridDim.x) {
            const int next = tile + gridDim.x;
            // the next tile's C rows: this warp's reads of the current ones are done
            __syncwarp();
            if (next < n_tiles) stage_tile(next);
            bool valid;
            int b, s;
            row_of(tile, valid, b, s);
            const bool wa_row = h == 0 && valid;
            const int src = wa_row ? lt.idx[(long long)t * lt.pitch + s] : 0;
            auto gather = [&]() {
                if (wa_row) {
                    cp_async<4>(smem_u32(&g_alpha[row]), m.half_alpha + src);
                    if (m.pol_m) cp_async<16>(smem_u32(&g_m[row]), m.pol_m + src);
                    else cp_async<4>(smem_u32(&g_m[row]), m.sqrt_flux + src);
                }
                cp_async_commit();
            };
            // ---- hidden layers 1 ..: accumulator -> bias, ReLU -> BF16 activations
            for (int l = 1; l < D; ++l) {
                if (!wait_bounded_spin(my_dfull, (uint32_t)(nd++) & 1u, abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                if (l == 1) gather();
                drain_layer(trow, ab, r_loc, c_beg, half, sbias + l * 256);
                tc_fence_before();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(my_afull);
            }
            if (!ok) break;
            // ---- output layer: accumulator -> registers, then the next tile's
            // h_1 (the accumulator columns are free again), then WA
            if (!wait_bounded_spin(my_dfull, (uint32_t)(nd++) & 1u, abort_flag, err)) { ok = false; break; }
            tc_fence_after();
            if (D == 1) gather();
            float y[8];
            if (h == 0) {
                uint32_t acc[16];
                tmem_ld16(trow, acc);
                tmem_wait_ld16(acc);
                const float* bo = sbias + D * 256;
#pragma unroll
                for (int i = 0; i < 8; ++i) y[i] = __uint_as_float(acc[i]) + bo[i];
            }
            tc_fence_before();
            cp_async_wait_all();
            if (next < n_tiles) start_tile(next);
            if (h == 0) {
                float mx = 0.f;
                if (valid) {
                    const float spec = expf(g_alpha[row] * ln_ratio);
                    const float4 gm = g_m[row];
                    float2* wb = wa + (long long)b * ncomp * wa_pitch + s;
                    if (!m.pol_m) {
                        const float w = gm.x * spec;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (c < ncomp) {
                                const float2 v = make_float2(w * y[2 * c], w * y[2 * c + 1]);
                                __stcs(wb + (long long)c * wa_pitch, v);
                                mx = fmaxf(mx, hypotf(v.x, v.y));
                            }
                    } else {  // two axes per feed: z = A M (eq. "fullz")
#pragma unroll
                        for (int c = 0; c < 4; c += 2)
                            if (c + 1 < ncomp) {
                                float2 z0, z1;
                                apply_sky_sqrt(make_float2(y[2 * c], y[2 * c + 1]),
                                               make_float2(y[2 * c + 2], y[2 * c + 3]), gm, spec, z0, z1);
                                __stcs(wb + (long long)c * wa_pitch, z0);
                                __stcs(wb + (long long)(c + 1) * wa_pitch, z1);
                                mx = fmaxf(mx, fmaxf(hypotf(z0.x, z0.y), hypotf(z1.x, z1.y)));
                            }
                    }
                }
                for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
                if (lane == 0 && mx > 0.f) atomicMax(reinterpret_cast<int*>(amax), __float_as_int(mx));
            }
        }
        cp_async_wait_all();
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

bool make_wmap(CUtensorMap* map, const void* base, int kin, int rows, int box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kin, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kin * 2};
    cuuint32_t box[2] = {KP, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t src_first_smem(int F, int H) { return sizeof(float) * ((size_t)2 * F * SRC_BLK + (size_t)SRC_BLK * (H + 4)); }

SrcArgs src_args(const MlpTcArgs& a) {
    SrcArgs s{};
    s.F = a.F; s.H = a.H; s.d0p = a.d0p; s.nu_mid = a.nu_mid; s.nu_half = a.nu_half; s.Bf = a.Bf;
    s.w0 = a.pb + a.off_w[0];
    return s;
}

}  // namespace

bool mlp_tc_supported(int F, int E, int H, int depth, int d0p, int n_out) {
    return (H == 128 || H == 256) && depth >= 1 && depth <= MAXL && d0p <= 256 && d0p % 16 == 0 && F % 8 == 0 &&
           E % 8 == 0 && n_out <= 8 && 2 * F + E <= d0p && F <= MAXF && get_encode() != nullptr;
}

cudaError_t mlp_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_wa, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_src_first, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)src_first_smem(MAXF, 256));
    return e;
}

long long mlp_tc_first_floats(int H, long long max_live) {
    return (max_live + SRC_BLK - 1) / SRC_BLK * SRC_BLK * H;
}

cudaError_t launch_mlp_beam_first(const MlpTcArgs& a, cudaStream_t st, long long* launches) {
    if (!mlp_tc_supported(a.F, a.E, a.H, a.depth, a.d0p, a.n_out) || !a.C || a.n_beam <= 0) return cudaErrorInvalidValue;
    k_beam_first<<<a.n_beam, a.H, 0, st>>>(src_args(a), a.E, a.p, a.off_b[0], a.off_emb, a.C);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_mlp_wa_tc(const MlpTcArgs& a, const Model& m, LiveTables lt, int t, int K, float nu,
                             float ln_ratio, float2* wa_slot, long long wa_pitch, float* amax, int* d_err, int n_sms,
                             cudaStream_t st, long long* launches) {
    if (K <= 0 || a.n_beam <= 0) return cudaSuccess;
    if (!mlp_tc_supported(a.F, a.E, a.H, a.depth, a.d0p, a.n_out) || !a.P || !a.C ||
        reinterpret_cast<uintptr_t>(a.pb + a.off_w[0]) % 16 != 0)
        return cudaErrorInvalidValue;
    Maps maps{};
    for (int l = 1; l <= a.depth; ++l) {
        const int rows = l == a.depth ? 8 : a.H;
        if (!make_wmap(&maps.w[l], a.pb + a.off_w[l], a.H, rows, rows)) return cudaErrorInvalidValue;
    }
    Net net{};
    net.H = a.H; net.depth = a.depth; net.n_beam = a.n_beam; net.n_out = a.n_out;
    net.p = a.p;
    for (int l = 0; l <= a.depth; ++l) net.off_b[l] = a.off_b[l];
    net.P = a.P;
    net.C = a.C;
    // P of this instance's live sources, then the rows of every beam
    const int n_blk = (K + SRC_BLK - 1) / SRC_BLK;
    k_src_first<<<n_blk, 256, src_first_smem(a.F, a.H), st>>>(src_args(a), lt, t, K, nu, a.P);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n_tiles = (long long)n_blk * ((a.n_beam + 7) / 8);
    if (n_tiles > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    const int grid = (int)std::max(1ll, std::min((long long)n_sms, n_tiles));
    k_mlp_wa<<<grid, THREADS, SMEM_BYTES, st>>>(maps, net, m, lt, t, K, ln_ratio, wa_slot, wa_pitch, amax, d_err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
