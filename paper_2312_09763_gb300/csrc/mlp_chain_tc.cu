// mlp_chain_tc.cu -- one launch for every row-local step of a training batch
// of the learned beam on the sm_103a tensor cores: the Fourier features, the
// hidden layers, the output layer with the loss and dL/dy, the input
// gradients back through the layers, and the embedding gradient.  The network
// and the loss are defined in mlp.cu; this kernel computes, for 128 rows at a
// time,
//   x0 = f(sample)                  (features: sin / cos of 2 pi B x, embedding)
//   h_l = relu(W_l h_{l-1} + b_l)   l = 0 .. D-1 (h_{-1} = x0)
//   y = W_out h_{D-1} + b_out,  r = y - target,  dL/dy = gscale r, loss += r.r
//   dz_{D-1} = (dL/dy W_out) * [h_{D-1} > 0]
//   dz_{l-1} = (dz_l W_l) * [h_{l-1} > 0]      l = D-1 .. 1
//   dL/de_a += (dz_0 W_0)[embedding columns]   (summed per beam a)
// and stores x0, every h_l, dL/dy and every dz_l batch-major for the weight
// gradients dW_l = dz_l^T h_{l-1}, which are products over the whole batch and
// run afterwards (mlp_train_tc.cu).
//
// A step is one product D[128][N] = A[128][K] B[N][K]^T with A the 128-row
// activation panels in shared memory (64 BF16 columns per 16 KB panel,
// 128-byte swizzle) and B the step's BF16 weights (W_l, W_out, W_out^T, W_l^T)
// streamed by TMA in 64-column panels through a ring.  One persistent CTA per
// SM walks 128-row tiles.  Warp 0 streams the weight panels, warp 1 owns TMEM
// and issues the MMAs (M = 128, N <= 256, K = 16) into two 256-column
// accumulators in turn, warp 2 stores each step's completed input panels to
// global memory with TMA (x0, h_l or dz_l), and warps 3-18 (four per TMEM lane
// quadrant; thread = one row and 16 columns of every 64-column panel) drain
// each step's accumulator through its epilogue back into the activation
// panels, panel by panel: the MMAs of step s + 1 start on panel 0 while the
// epilogue of step s still writes the later panels.  A step's epilogue
// overwrites the panels once the stores have read them.  The ReLU masks of
// the forward layers stay in shared memory as bits for the backward steps
// (the same thread reads back its own bits), so the backward pass reads no
// activations.
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

constexpr int TM = 128;                      // rows per tile (one TMEM lane each)
constexpr int KP = 64;                       // columns per activation / weight panel (128 B of BF16)
constexpr int MAXL = kChainMaxLayers;
constexpr int MAXS = 2 * MAXL + 2;           // steps per tile at most
constexpr int A_PANEL = TM * 128;            // 16 KB
constexpr int SMEM_ACT = 4 * A_PANEL;        // 64 KB: up to 256 columns
constexpr int W_SLOT = 256 * 128;            // 32 KB: a weight panel of up to 256 rows
constexpr int NEPI = 16;                     // epilogue warps
constexpr int THREADS = (3 + NEPI) * 32;    // producer, MMA, storer, epilogue
constexpr int TMEM_COLS = 512;               // two 256-column accumulators
constexpr int MAX_SMEM = 227 * 1024;

enum StepKind : int { K_RELU = 0, K_LOSS = 1, K_MASK = 2, K_EMB = 3 };

struct Maps {
    CUtensorMap w[MAXS];   // B operand of step s
    CUtensorMap st[MAXS];  // destination of step s's input panels (if store[s])
};

struct Job {
    int M, n_tiles, ns, nslot;
    int D, H, F, E, d0p, n_out;
    float nu_mid, nu_half, gscale;
    int K[MAXS], N[MAXS], wrows[MAXS], store[MAXS], kind[MAXS], lay[MAXS];
    const float* p;
    long long off_b[MAXL + 1];
    long long off_emb;
    const float* Bf;
    const int* ant;
    const float *az, *za, *nu, *T;
    bf16* dY;
    double* loss;
    float* gemb;
};

// Shared memory past the activation panels and the weight ring: the mask
// bits [D][4 panels][4 column groups][128 rows] (16 bits), the biases
// [D + 1][256], the Fourier matrix [F] as float4, then the barriers.
// the tensor maps and the job travel as kernel parameters: keep them inside
// the classic 4 KB parameter space
static_assert(sizeof(Maps) + sizeof(Job) + sizeof(int*) <= 4096, "kernel parameters over 4 KB");

__host__ __device__ constexpr int mask_off(int nslot) { return SMEM_ACT + nslot * W_SLOT; }
__host__ __device__ constexpr int bias_off(int nslot, int D) { return mask_off(nslot) + D * 4 * 4 * TM * 2; }
__host__ __device__ constexpr int fb_off(int nslot, int D) { return bias_off(nslot, D) + (D + 1) * 256 * 4; }
__host__ __device__ constexpr int bar_off(int nslot, int D, int F) { return fb_off(nslot, D) + F * 16; }
__host__ __device__ constexpr int smem_bytes(int nslot, int D, int F) {
    return 1024 + bar_off(nslot, D, F) + (2 * nslot + 9) * 8 + 16;
}

// Shared-memory address of the 16-byte chunk holding columns [8 j, 8 j + 8)
// of activation panel col / 64, row r (128-byte swizzle: chunk j ^ (r & 7)).
__device__ __forceinline__ uint32_t a_chunk(uint32_t a_base, int r, int col) {
    const int panel = col / KP, j = (col % KP) / 8;
    return a_base + panel * A_PANEL + r * 128 + ((j ^ (r & 7)) << 4);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_global_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// max(lo, 0) in the low half, max(hi, 0) in the high half, rounded to BF16.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
// Registers of a second tcgen05.ld: no use of them may move above the
// tcgen05.wait::ld that precedes this point.
__device__ __forceinline__ void keep_after_wait16(uint32_t (&r)[16]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

// Sum of x over the warp's 32 lanes for 16 columns at once: afterwards lane l
// holds the sum of column l & 15.
__device__ __forceinline__ float column_sums16(float (&x)[16], int lane) {
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = up ? x[i] : x[i + w];
            const float keep = up ? x[i + w] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return x[0] + __shfl_xor_sync(0xffffffffu, x[0], 16);
}

// What an epilogue thread needs to write the activation panels and release
// them (passed by value: no addresses of locals are taken in this kernel).
struct Epi {
    uint32_t act;     // activation panels
    uint32_t afull0;  // barrier "panel p of the next step's input written" at afull0 + 8 p
    int r, cg, lane;  // row of the tile, column group, lane
    const float4* sB;
};

__device__ __forceinline__ void arrive_panel(const Epi e, int p) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (e.lane == 0) mbar_arrive(e.afull0 + 8u * (uint32_t)p);
}

// One row's sample: beam and the network's inputs x.
struct Row {
    int valid, a;
    float x0, x1, x2;
};

__device__ __forceinline__ Row load_row(const Job& j, int tile, int r) {
    Row w{0, 0, 0.f, 0.f, 0.f};
    const long long m = (long long)tile * TM + r;
    if (tile < j.n_tiles && m < j.M) {
        w.valid = 1;
        w.a = j.ant[m];
        w.x0 = j.az[m] * 0.15915494309189535f;  // az / 2 pi
        w.x1 = j.za[m] * 0.63661977236758134f;  // za / (pi / 2)
        w.x2 = (j.nu[m] - j.nu_mid) / j.nu_half;
    }
    return w;
}

// Features of one row, [sin 2 pi B x, cos 2 pi B x, e_a, 0 ...], into the
// activation panels; every panel released.  The row's four threads (column
// groups cg) share it by 8-column chunks: chunk k of the sines and chunk k of
// the cosines (one sincos per phase) for k = cg, cg + 4, ..., then the
// embedding and zero chunks likewise.  The phase is reduced to [-1/2, 1/2]
// turn, where the fast sine and cosine are accurate to ~1e-6, far below the
// BF16 rounding of the features.
__device__ __forceinline__ void write_features(const Job& j, const Epi e, const Row w) {
    for (int k = e.cg; k < j.F / 8; k += 4) {
        float sv[8], cv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 b = e.sB[8 * k + i];
            float ph = b.x * w.x0 + b.y * w.x1 + b.z * w.x2;
            ph -= rintf(ph);
            __sincosf(6.283185307179586f * ph, &sv[i], &cv[i]);
            if (!w.valid) sv[i] = cv[i] = 0.f;
        }
        st_shared_v4(a_chunk(e.act, e.r, 8 * k), pack_bf16(sv[0], sv[1]), pack_bf16(sv[2], sv[3]),
                     pack_bf16(sv[4], sv[5]), pack_bf16(sv[6], sv[7]));
        st_shared_v4(a_chunk(e.act, e.r, j.F + 8 * k), pack_bf16(cv[0], cv[1]), pack_bf16(cv[2], cv[3]),
                     pack_bf16(cv[4], cv[5]), pack_bf16(cv[6], cv[7]));
    }
    for (int k = 2 * j.F / 8 + e.cg; k < j.d0p / 8; k += 4) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ce = 8 * k + i - 2 * j.F;  // embedding column
            v[i] = w.valid && ce < j.E ? j.p[j.off_emb + (long long)w.a * j.E + ce] : 0.f;
        }
        st_shared_v4(a_chunk(e.act, e.r, 8 * k), pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                     pack_bf16(v[6], v[7]));
    }
    for (int p = 0; p < 4; ++p) arrive_panel(e, p);
}

// One 16-column chunk of a hidden layer's accumulator: bias and ReLU into the
// activation panel, and the chunk's 16 mask bits (the returned value).
__device__ __forceinline__ uint32_t emit_relu(const Epi e, int c, const float* bias, const uint32_t (&a)[16]) {
    uint32_t h[8];
    uint32_t bits = 0;
    const float4* b4 = reinterpret_cast<const float4*>(bias + c);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 b = b4[q];
        h[2 * q] = relu_bf16x2(__uint_as_float(a[4 * q]) + b.x, __uint_as_float(a[4 * q + 1]) + b.y);
        h[2 * q + 1] = relu_bf16x2(__uint_as_float(a[4 * q + 2]) + b.z, __uint_as_float(a[4 * q + 3]) + b.w);
    }
    // a ReLU output is positive exactly when its BF16 bits, sign cleared, are
    // not zero: adding 0x7FFF to each 16-bit half then sets its top bit (no
    // carry between the halves), which lands at bit 2k (low half) or 16 + 2k
    // (high half) of `lo`
    uint32_t lo = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) lo |= (((h[k] & 0x7FFF7FFFu) + 0x7FFF7FFFu) & 0x80008000u) >> (15 - 2 * k);
    bits = (lo & 0x5555u) | ((lo >> 15) & 0xAAAAu);
    st_shared_v4(a_chunk(e.act, e.r, c), h[0], h[1], h[2], h[3]);
    st_shared_v4(a_chunk(e.act, e.r, c + 8), h[4], h[5], h[6], h[7]);
    return bits;
}

// One 16-column chunk of an input gradient, masked by the forward layer's
// ReLU bits, into the activation panel.
__device__ __forceinline__ void emit_mask(const Epi e, int c, uint32_t bits, const uint32_t (&a)[16]) {
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        h[k] = pack_bf16((bits >> (2 * k)) & 1u ? __uint_as_float(a[2 * k]) : 0.f,
                         (bits >> (2 * k + 1)) & 1u ? __uint_as_float(a[2 * k + 1]) : 0.f);
    st_shared_v4(a_chunk(e.act, e.r, c), h[0], h[1], h[2], h[3]);
    st_shared_v4(a_chunk(e.act, e.r, c + 8), h[4], h[5], h[6], h[7]);
}

__global__ void __launch_bounds__(THREADS, 1)
k_mlp_chain(const __grid_constant__ Maps maps, const __grid_constant__ Job j, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int NSL = j.nslot, D = j.D;
    const uint32_t act = smem_u32(smem);
    const uint32_t ring = act + SMEM_ACT;
    uint16_t* smask = reinterpret_cast<uint16_t*>(smem + mask_off(NSL));
    float* sbias = reinterpret_cast<float*>(smem + bias_off(NSL, D));
    float4* sB = reinterpret_cast<float4*>(smem + fb_off(NSL, D));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + bar_off(NSL, D, j.F));
    // barriers: wfull[NSL], wfree[NSL], afull[4], dfull[2], tempty[2], sdone
    const uint32_t b0 = smem_u32(bars);
    const uint32_t WFULL = b0, WFREE = b0 + 8u * NSL, AFULL = b0 + 16u * NSL, DFULL = AFULL + 32u, TEMPTY = AFULL + 48u,
                   SDONE = AFULL + 64u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSL + 9);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = j.ns;

    for (int l = 0; l <= D; ++l) {
        const int n = l == D ? j.n_out : j.H;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) sbias[l * 256 + i] = i < n ? j.p[j.off_b[l] + i] : 0.f;
    }
    for (int f = threadIdx.x; f < j.F; f += blockDim.x)
        sB[f] = make_float4(j.Bf[3 * f], j.Bf[3 * f + 1], j.Bf[3 * f + 2], 0.f);
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSL; ++i) { mbar_init(WFULL + 8u * i, 1); mbar_init(WFREE + 8u * i, 1); }
        for (int p = 0; p < 4; ++p) mbar_init(AFULL + 8u * p, NEPI);
        for (int b = 0; b < 2; ++b) { mbar_init(DFULL + 8u * b, 1); mbar_init(TEMPTY + 8u * b, NEPI); }
        mbar_init(SDONE, 1);
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
        // ---- weight panels of every step, in step order, through the ring
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint64_t keep = policy_evict_last();  // the weights stay in L2 for every tile
            for (int tile = blockIdx.x; tile < j.n_tiles && ok; tile += gridDim.x)
                for (int s = 0; s < NS && ok; ++s) {
                    const int np = (j.K[s] + KP - 1) / KP;
                    for (int p = 0; p < np; ++p, ++it) {
                        const int sl = it % NSL;
                        if (!wait_bounded_spin(WFREE + 8u * sl, ((uint32_t)(it / NSL) & 1u) ^ 1u, abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(WFULL + 8u * sl, (uint32_t)(j.wrows[s] * 128));
                        tma_load_2d_hint(ring + sl * W_SLOT, &maps.w[s], p * KP, 0, WFULL + 8u * sl, keep);
                    }
                }
        }
    } else if (warp == 1) {
        // ---- MMAs
        if (lane == 0) {
            int it = 0, g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < j.n_tiles && ok; tile += gridDim.x)
                for (int s = 0; s < NS && ok; ++s, ++g) {
                    const int buf = g & 1;
                    if (!wait_bounded_spin(TEMPTY + 8u * buf, ((uint32_t)(g >> 1) & 1u) ^ 1u, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int K = j.K[s], np = (K + KP - 1) / KP;
                    const uint32_t id = idesc_f16(false, TM, j.N[s]);
                    const uint32_t d = tmem + (uint32_t)(buf * 256);
                    for (int p = 0; p < np; ++p, ++it) {
                        // panel p of this step's input, written by the previous epilogue
                        if (!wait_bounded_spin(AFULL + 8u * p, (uint32_t)g & 1u, abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int sl = it % NSL;
                        if (!wait_bounded_spin(WFULL + 8u * sl, (uint32_t)(it / NSL) & 1u, abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int ks = min(KP, K - p * KP) / 16;
                        for (int kk = 0; kk < ks; ++kk)
                            tc_mma(d, sdesc(act + p * A_PANEL + kk * 32), sdesc(ring + sl * W_SLOT + kk * 32), id,
                                   (p | kk) != 0 ? 1u : 0u);
                        tc_commit(WFREE + 8u * sl);
                    }
                    if (!ok) break;
                    tc_commit(DFULL + 8u * buf);
                }
        }
    } else if (warp == 2) {
        // ---- TMA stores of each step's input panels (x0, h_l, dz_l) as they
        // complete; a step's epilogue overwrites the panels only once the
        // stores have read them (sdone, once per step)
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < j.n_tiles && ok; tile += gridDim.x)
                for (int s = 0; s < NS && ok; ++s, ++g) {
                    const int np = (j.K[s] + KP - 1) / KP;
                    for (int p = 0; p < np; ++p) {
                        if (!wait_bounded_spin(AFULL + 8u * p, (uint32_t)g & 1u, abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        if (j.store[s]) tma_store_2d(&maps.st[s], p * KP, tile * TM, act + p * A_PANEL);
                    }
                    if (!ok) break;
                    if (j.store[s]) {
                        bulk_commit();
                        bulk_wait_read_all();
                    }
                    mbar_arrive(SDONE);
                }
            bulk_commit();
            bulk_wait_all();
        }
    } else {
        // ---- epilogue warps: TMEM lane quadrant q, columns [16 cg, 16 cg + 16)
        // of every 64-column panel; thread = row r of the tile
        const int q = warp & 3, cg = (warp - 3) >> 2;
        const int r = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const Epi e{act, AFULL, r, cg, lane, sB};
        uint16_t* my_mask = smask + cg * TM + r;  // bits of layer l, panel p at my_mask[(l * 4 + p) * 4 * TM]
        bool ok = true;
        int g = 0;
        int tile = blockIdx.x;
        Row cur = load_row(j, tile, r);
        if (tile < j.n_tiles) write_features(j, e, cur);
        for (; tile < j.n_tiles && ok; tile += gridDim.x) {
            const long long m = (long long)tile * TM + r;
            // read ahead: the next tile's sample (its features are written at this
            // tile's last step; its embedding row fetched into L1 now) and this
            // row's targets (the loss step)
            const Row nxt = load_row(j, tile + gridDim.x, r);
            if (nxt.valid) asm volatile("prefetch.global.L1 [%0];" ::"l"(j.p + j.off_emb + (long long)nxt.a * j.E));
            float tg0 = 0.f, tg1 = 0.f;
            if (cur.valid && 2 * cg < j.n_out) {
                tg0 = j.T[m * j.n_out + 2 * cg];
                tg1 = j.T[m * j.n_out + 2 * cg + 1];
            }
            for (int s = 0; s < NS; ++s, ++g) {
                const int buf = g & 1;
                if (!wait_bounded(DFULL + 8u * buf, (uint32_t)(g >> 1) & 1u, abort_flag, err, kTimeoutNs, 1000u) ||
                    !wait_bounded_spin(SDONE, (uint32_t)g & 1u, abort_flag, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tl + (uint32_t)(buf * 256);
                const int kind = j.kind[s], l = j.lay[s];
                if (kind == K_RELU || kind == K_MASK) {
                    // the accumulator's H columns two panels at a time, each panel
                    // released as soon as it is written
                    const int np = j.H / KP;
                    const float* bias = sbias + l * 256;
                    for (int p = 0; p < np; p += 2) {
                        uint32_t acc0[16], acc1[16];
                        const int c0 = p * KP + 16 * cg;
                        tmem_ld16(tb + c0, acc0);
                        if (p + 1 < np) tmem_ld16(tb + c0 + KP, acc1);
                        tmem_wait_ld16(acc0);
                        if (p + 1 < np) keep_after_wait16(acc1);
                        if (kind == K_RELU) my_mask[(l * 4 + p) * 4 * TM] = (uint16_t)emit_relu(e, c0, bias, acc0);
                        else emit_mask(e, c0, my_mask[(l * 4 + p) * 4 * TM], acc0);
                        arrive_panel(e, p);
                        if (p + 1 < np) {
                            if (kind == K_RELU)
                                my_mask[(l * 4 + p + 1) * 4 * TM] = (uint16_t)emit_relu(e, c0 + KP, bias, acc1);
                            else emit_mask(e, c0 + KP, my_mask[(l * 4 + p + 1) * 4 * TM], acc1);
                            arrive_panel(e, p + 1);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(TEMPTY + 8u * buf);
                    for (int p = np; p < 4; ++p) arrive_panel(e, p);
                } else if (kind == K_LOSS) {
                    // warp cg: outputs 2 cg and 2 cg + 1 (component cg), residual
                    // against the target, dL/dy into column 2 cg of panel 0 (the
                    // next step's K = 16 input) and into dY
                    float lsum = 0.f;
                    if (2 * cg < j.n_out) {
                        uint32_t a2[2];
                        tmem_ld2(tb + 2 * cg, a2);
                        tmem_wait_ld2(a2);
                        float g0 = 0.f, g1 = 0.f;
                        if (cur.valid) {
                            const float r0 = __uint_as_float(a2[0]) + sbias[D * 256 + 2 * cg] - tg0;
                            const float r1 = __uint_as_float(a2[1]) + sbias[D * 256 + 2 * cg + 1] - tg1;
                            lsum = r0 * r0 + r1 * r1;
                            g0 = j.gscale * r0;
                            g1 = j.gscale * r1;
                        }
                        const uint32_t h = pack_bf16(g0, g1);
                        asm volatile("st.shared.b32 [%0], %1;" ::"r"(a_chunk(act, r, 2 * cg) + 4u * (uint32_t)cg),
                                     "r"(h)
                                     : "memory");
                        if (cur.valid) *reinterpret_cast<uint32_t*>(j.dY + m * 64 + 2 * cg) = h;
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(TEMPTY + 8u * buf);
                    for (int p = 0; p < 4; ++p) arrive_panel(e, p);
                    if (2 * cg < j.n_out) {
                        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
                        if (lane == 0 && lsum != 0.f) atomicAdd(j.loss, (double)lsum);
                    }
                } else {
                    // K_EMB: the next tile's features first (the next step reads
                    // them; it accumulates in the other TMEM buffer), then the
                    // embedding gradient, rows of one beam summed over the warp
                    // before the atomic add (each beam's rows lie together)
                    if (tile + (int)gridDim.x < j.n_tiles) write_features(j, e, nxt);
                    for (int p = 0; p < 4; ++p) {
                        const int c = p * KP + 16 * cg;
                        if (c >= j.E) continue;
                        uint32_t a[16];
                        tmem_ld16(tb + c, a);
                        tmem_wait_ld16(a);
                        const int nv = min(16, j.E - c);
                        const int ab = cur.valid ? cur.a : -1;
                        unsigned rem = __ballot_sync(0xffffffffu, cur.valid);
                        while (rem) {
                            const int al = __shfl_sync(0xffffffffu, ab, __ffs(rem) - 1);
                            const unsigned grp = __ballot_sync(0xffffffffu, ab == al);
                            float x[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) x[i] = ab == al ? __uint_as_float(a[i]) : 0.f;
                            const float cs = column_sums16(x, lane);
                            if (lane < nv) atomicAdd(j.gemb + (long long)al * j.E + c + lane, cs);
                            rem &= ~grp;
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(TEMPTY + 8u * buf);
                }
                if (*abort_flag) {
                    ok = false;
                    break;
                }
            }
            cur = nxt;
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

// 2D BF16 tensor (inner, rows) of row pitch ld elements with boxes of 64
// inner elements x box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, long long inner, long long rows, long long ld, int box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc || ((uintptr_t)base & 15) || (ld * 2) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {KP, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int ring_slots(int D, int F) {
    for (int n = 4; n >= 2; --n)
        if (smem_bytes(n, D, F) <= MAX_SMEM) return n;
    return 0;
}

}  // namespace

bool mlp_chain_supported(int F, int E, int H, int depth, int d0p, int n_out, int M) {
    return H % KP == 0 && H >= KP && H <= 256 && depth >= 1 && depth <= MAXL && d0p % 16 == 0 && d0p >= KP &&
           d0p <= 256 && F >= 1 && F <= 128 && F % 8 == 0 && E >= 1 && 2 * F + E <= d0p && n_out >= 1 &&
           n_out <= 8 && M >= TM && ring_slots(depth, F) >= 2 && get_encode() != nullptr;
}

cudaError_t mlp_chain_init() {
    return cudaFuncSetAttribute(k_mlp_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
}

cudaError_t launch_mlp_chain_tc(const ChainArgs& a, int n_sms, int* d_err, cudaStream_t st, long long* launches) {
    if (!mlp_chain_supported(a.F, a.E, a.H, a.depth, a.d0p, a.n_out, a.M)) return cudaErrorInvalidValue;
    const int D = a.depth, H = a.H;
    const int erows = (a.E + 15) / 16 * 16;
    Maps maps{};
    Job j{};
    j.M = a.M;
    j.n_tiles = (a.M + TM - 1) / TM;
    j.ns = 2 * D + 2;
    j.nslot = ring_slots(D, a.F);
    j.D = D; j.H = H; j.F = a.F; j.E = a.E; j.d0p = a.d0p; j.n_out = a.n_out;
    j.nu_mid = a.nu_mid; j.nu_half = a.nu_half; j.gscale = a.gscale;
    j.p = a.p;
    for (int l = 0; l <= D; ++l) j.off_b[l] = a.off_b[l];
    j.off_emb = a.off_emb;
    j.Bf = a.Bf;
    j.ant = a.ant; j.az = a.az; j.za = a.za; j.nu = a.nu; j.T = a.T;
    j.dY = a.dY; j.loss = a.loss; j.gemb = a.gemb;
    bool ok = true;
    // forward: step l multiplies by W_l ([H][kin_l]) and stores its input (x0 or h_{l-1})
    for (int l = 0; l < D; ++l) {
        const int kin = l == 0 ? a.d0p : H;
        j.K[l] = kin; j.N[l] = H; j.wrows[l] = H; j.kind[l] = K_RELU; j.lay[l] = l; j.store[l] = 1;
        ok = ok && make_map(&maps.w[l], a.w[l], kin, H, kin, H);
        ok = ok && (l == 0 ? make_map(&maps.st[l], a.X0, a.d0p, a.M, a.d0p, TM)
                           : make_map(&maps.st[l], a.Hs[l - 1], H, a.M, H, TM));
    }
    // output layer and loss (W_out padded to 16 rows); stores h_{D-1}
    j.K[D] = H; j.N[D] = 16; j.wrows[D] = 16; j.kind[D] = K_LOSS; j.lay[D] = D; j.store[D] = 1;
    ok = ok && make_map(&maps.w[D], a.wout16, H, 16, H, 16) && make_map(&maps.st[D], a.Hs[D - 1], H, a.M, H, TM);
    // dL/dy times W_out (W_out^T [H][64], K = 16), masked by h_{D-1}
    j.K[D + 1] = 16; j.N[D + 1] = H; j.wrows[D + 1] = H; j.kind[D + 1] = K_MASK; j.lay[D + 1] = D - 1;
    j.store[D + 1] = 0;
    ok = ok && make_map(&maps.w[D + 1], a.woutT, 64, H, 64, H);
    // dz_l times W_l (W_l^T [H][H]), masked by h_{l-1}; stores dz_l
    for (int l = D - 1; l >= 1; --l) {
        const int s = 2 * D + 1 - l;
        j.K[s] = H; j.N[s] = H; j.wrows[s] = H; j.kind[s] = K_MASK; j.lay[s] = l - 1; j.store[s] = 1;
        ok = ok && make_map(&maps.w[s], a.wt[l], H, H, H, H) && make_map(&maps.st[s], a.dZs[l], H, a.M, H, TM);
    }
    // dz_0 times the embedding rows of W_0^T; stores dz_0
    {
        const int s = 2 * D + 1;
        j.K[s] = H; j.N[s] = erows; j.wrows[s] = erows; j.kind[s] = K_EMB; j.lay[s] = 0; j.store[s] = 1;
        ok = ok && make_map(&maps.w[s], a.wt[0] + (long long)2 * a.F * H, H, erows, H, erows) &&
             make_map(&maps.st[s], a.dZs[0], H, a.M, H, TM);
    }
    if (!ok) return cudaErrorInvalidValue;
    // as few CTAs as keep the most tiles any CTA walks (the others' SMs stay free)
    const int per_cta = (j.n_tiles + std::max(1, n_sms) - 1) / std::max(1, n_sms);
    const int grid = std::max(1, (j.n_tiles + per_cta - 1) / per_cta);
    k_mlp_chain<<<grid, THREADS, smem_bytes(j.nslot, D, a.F), st>>>(maps, j, d_err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
