// mlp_tc.cu -- the learned beam's forward pass on the sm_103a tensor cores,
// fused with the beam-times-flux step of the simulator: for every row
// (antenna beam b, live source s) of one instance it builds the network's
// input features, runs the hidden layers and the output layer with
// tcgen05.mma, and writes WA[b][comp][s] = sqrt(I_s(nu)) A^{pk}_b(s) (or,
// for a polarised sky, A M with the coherency square root, eq. "fullz") --
// Algorithm 2 step (ii) of arXiv:2312.09763 with the network in place of the
// interpolation of Sec. 2.4.
//
// The network (mlp.cu): x = (az / 2 pi, za / (pi/2), (nu - nu_mid) / nu_half),
// f = [sin(2 pi B x), cos(2 pi B x), e_b, 0...] (d0p columns), h_l = relu(W_l
// h_{l-1} + b_l) for the hidden layers, y = W_out h + b_out.  Operands are
// BF16, accumulation FP32 in TMEM, as in the training kernels.
//
// One persistent CTA per SM walks 256-row tiles made of two 128-row
// sub-tiles with their own activation panels and TMEM accumulators (columns 0
// and 256), so that every weight panel feeds the MMAs of both.  Warp 0 streams
// the weight panels (64 input columns x H rows, 128-byte swizzle) with TMA
// through a ring of two slots; warp 1 owns TMEM and issues the MMAs (M = 128,
// N = H, K = 16); warps 2..17 (one per TMEM lane quadrant, sub-tile and half
// of the columns) write the features, drain each layer's accumulator through
// bias and ReLU back into the shared-memory activation panels, and write WA
// from the output layer.  Every mbarrier wait is bounded (tc.cuh).
#include <cuda_bf16.h>

#include <algorithm>
#include "common.cuh"
#include "tc.cuh"

namespace mv {
namespace {

using namespace tc;

constexpr int TM = 128;          // rows per sub-tile (one TMEM accumulator)
constexpr int TILE = 2 * TM;     // rows per tile: two sub-tiles share every weight panel
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
constexpr int SMEM_FB = MAXF * 16;                // B as float4 rows
constexpr int NEPI = 16;                          // epilogue warps: four per TMEM lane quadrant
// per-row values gathered ahead of use with cp.async: the next tile's (az, za)
// for every epilogue thread, and (m00, Re m10, Im m10, m11) or (flux, 0, 0, 0)
// plus the spectral index of this tile's sources for the WA writers
constexpr int SMEM_GATHER = NEPI * 32 * 8 + TILE * 16 + TILE * 4;
constexpr int SMEM_BYTES = SMEM_A + SMEM_W + SMEM_O + SMEM_BIAS + SMEM_FB + SMEM_GATHER + 256 + 1024;
constexpr int THREADS = (2 + NEPI) * 32;

struct Maps {
    CUtensorMap w[MAXL + 1];  // hidden layers, then the output layer
};

struct Net {
    int F, E, H, depth, d0p, n_beam, n_out;
    float nu_mid, nu_half;
    const float* p;  // FP32 parameters (biases, embedding)
    long long off_b[MAXL + 1];
    long long off_emb;
    const float* Bf;  // [F][3]
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

// Registers of a second tcgen05.ld: no use of them may move above the
// tcgen05.wait::ld that precedes this point.
__device__ __forceinline__ void keep_after_wait16(uint32_t (&r)[16]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

// Ampere-style asynchronous global -> shared copies of 4, 8 or 16 bytes.
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t saddr, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr), "l"(g), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(THREADS, 1)
k_mlp_wa(const __grid_constant__ Maps maps, const __grid_constant__ Net net, Model m, LiveTables lt, int t, int K,
         float nu, float ln_ratio, float2* __restrict__ wa, long long wa_pitch, float* __restrict__ amax,
         int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t a_base = smem_u32(smem);
    const uint32_t w_base = a_base + SMEM_A;
    const uint32_t o_base = w_base + SMEM_W;
    float* sbias = reinterpret_cast<float*>(smem + SMEM_A + SMEM_W + SMEM_O);  // [layer][256]
    float4* sB = reinterpret_cast<float4*>(smem + SMEM_A + SMEM_W + SMEM_O + SMEM_BIAS);  // [F] (B_f0, B_f1, B_f2, 0)
    uint8_t* sgather = smem + SMEM_A + SMEM_W + SMEM_O + SMEM_BIAS + SMEM_FB;
    float2* g_azza = reinterpret_cast<float2*>(sgather);                         // [epilogue thread]
    float4* g_m = reinterpret_cast<float4*>(sgather + NEPI * 32 * 8);            // [row of the tile]
    float* g_alpha = reinterpret_cast<float*>(sgather + NEPI * 32 * 8 + TILE * 16);  // [row of the tile]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sgather + SMEM_GATHER);
    // wfull[NSLOT], wfree[NSLOT], afull, dfull, ofull
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSLOT + 3);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    auto wfull = [&](int i) { return smem_u32(&bars[i]); };
    auto wfree = [&](int i) { return smem_u32(&bars[NSLOT + i]); };
    const uint32_t afull = smem_u32(&bars[2 * NSLOT]), dfull = smem_u32(&bars[2 * NSLOT + 1]),
                   ofull = smem_u32(&bars[2 * NSLOT + 2]);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = net.H, D = net.depth;
    const long long R = (long long)net.n_beam * K;
    const int n_tiles = (int)((R + TILE - 1) / TILE);
    const int w_panel = H * 128;
    auto panels = [&](int l) { return l == 0 ? (net.d0p + KP - 1) / KP : H / KP; };
    auto ksteps = [&](int l, int pnl) {  // 16-column MMA steps in panel pnl of layer l
        const int kin = l == 0 ? net.d0p : H;
        return min(KP, kin - pnl * KP) / 16;
    };

    // output-layer panels: rows 8..15 stay zero (the tensor map fills rows 0..7)
    for (int i = threadIdx.x; i < SMEM_O / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem + SMEM_A + SMEM_W)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int l = 0; l <= D; ++l) {
        const int n = l == D ? 8 : H;
        for (int i = threadIdx.x; i < n; i += blockDim.x) sbias[l * 256 + i] = net.p[net.off_b[l] + i];
    }
    for (int f = threadIdx.x; f < net.F; f += blockDim.x)
        sB[f] = make_float4(net.Bf[3 * f], net.Bf[3 * f + 1], net.Bf[3 * f + 2], 0.f);
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) { mbar_init(wfull(i), 1); mbar_init(wfree(i), 1); }
        mbar_init(afull, NEPI);
        mbar_init(dfull, 1);
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
            mbar_expect_tx(ofull, (uint32_t)((H / KP) * (O_PANEL / 2)));
            for (int pnl = 0; pnl < H / KP; ++pnl) tma_load_2d(o_base + pnl * O_PANEL, &maps.w[D], pnl * KP, 0, ofull);
            int it = 0;  // weight panels streamed so far (ring position)
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
                for (int l = 0; l < D && ok; ++l)
                    for (int pnl = 0; pnl < panels(l); ++pnl, ++it) {
                        const int sl = it % NSLOT;
                        if (!wait_bounded_spin(wfree(sl), ((uint32_t)(it / NSLOT) & 1u) ^ 1u, abort_flag, err)) { ok = false; break; }
                        mbar_expect_tx(wfull(sl), (uint32_t)w_panel);
                        tma_load_2d(w_base + sl * W_PANEL_MAX, &maps.w[l], pnl * KP, 0, wfull(sl));
                    }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id_hidden = idesc_f16(false, TM, H), id_out = idesc_f16(false, TM, 16);
            int it = 0;
            int na = 0;
            bool ok = wait_bounded_spin(ofull, 0u, abort_flag, err);
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int l = 0; l <= D && ok; ++l) {
                    if (!wait_bounded_spin(afull, (uint32_t)(na++) & 1u, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const bool out = l == D;
                    const int np = out ? H / KP : panels(l);
                    for (int pnl = 0; pnl < np; ++pnl) {
                        const int sl = it % NSLOT;
                        if (!out) {
                            if (!wait_bounded_spin(wfull(sl), (uint32_t)(it / NSLOT) & 1u, abort_flag, err)) { ok = false; break; }
                            tc_fence_after();
                        }
                        const uint32_t b0 = out ? o_base + pnl * O_PANEL : w_base + sl * W_PANEL_MAX;
                        const int ns = out ? KP / 16 : ksteps(l, pnl);
                        // both sub-tiles from the same weight panel (accumulators at columns 0 and 256)
                        for (int u = 0; u < 2; ++u)
                            for (int kk = 0; kk < ns; ++kk)
                                tc_mma(tmem + (uint32_t)(u * 256), sdesc(a_base + u * SUB_A + pnl * A_PANEL + kk * 32),
                                       sdesc(b0 + kk * 32), out ? id_out : id_hidden, (pnl | kk) != 0 ? 1u : 0u);
                        if (!out) {
                            tc_commit(wfree(sl));
                            ++it;
                        }
                    }
                    if (!ok) break;
                    tc_commit(dfull);
                }
            }
        }
    } else {
        // epilogue warps: lane quadrant q, sub-tile u, column half h
        const int q = warp & 3, u = ((warp - 2) >> 2) & 1, h = (warp - 2) >> 3;
        const int r_loc = q * 32 + lane;  // row within the sub-tile
        const int row = u * TM + r_loc;   // row within the tile
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(u * 256);
        const uint32_t ab = a_base + u * SUB_A;
        const int F = net.F, E = net.E;
        const int ncomp = net.n_out / 2;
        const uint32_t my_azza = smem_u32(&g_azza[threadIdx.x - 64]);
        int nd = 0;
        bool ok = true;
        // row of the network input in a tile: beam b, live source s
        auto row_of = [&](int tile, bool& valid, int& b, int& s) {
            const long long r = (long long)tile * TILE + row;
            valid = r < R;
            b = valid ? (int)(r / K) : 0;
            s = valid ? (int)(r % K) : 0;
        };
        // input features of this thread's row: chunks of 8 columns, chunk c by half c % 2
        auto features = [&](bool valid, int b, float2 azza) {
            const float x0 = azza.x * 0.15915494309189535f;   // az / 2 pi
            const float x1 = azza.y * 0.63661977236758134f;   // za / (pi / 2)
            const float x2 = (nu - net.nu_mid) / net.nu_half;
            for (int c8 = 8 * h; c8 < F; c8 += 16) {
                float sv[8], cv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 bf = sB[c8 + i];
                    float ph = bf.x * x0 + bf.y * x1 + bf.z * x2;
                    ph -= rintf(ph);
                    // |2 pi ph| <= pi: the fast sine and cosine are accurate to ~1e-6
                    // there, far below the BF16 rounding of the features
                    __sincosf(6.283185307179586f * ph, &sv[i], &cv[i]);
                    if (!valid) sv[i] = cv[i] = 0.f;
                }
                st_shared_v4(a_chunk(ab, r_loc, c8), pack_bf16(sv[0], sv[1]), pack_bf16(sv[2], sv[3]),
                             pack_bf16(sv[4], sv[5]), pack_bf16(sv[6], sv[7]));
                st_shared_v4(a_chunk(ab, r_loc, F + c8), pack_bf16(cv[0], cv[1]), pack_bf16(cv[2], cv[3]),
                             pack_bf16(cv[4], cv[5]), pack_bf16(cv[6], cv[7]));
            }
            const float* e = net.p + net.off_emb + (long long)b * E;
            for (int c8 = 8 * h; c8 < net.d0p - 2 * F; c8 += 16) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = valid && c8 + i < E ? e[c8 + i] : 0.f;
                st_shared_v4(a_chunk(ab, r_loc, 2 * F + c8), pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                             pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(afull);
        };
        // Per tile: the next tile's (az, za) and, for the WA writers (half 0),
        // the source index are requested at the start, the index's flux,
        // spectral index (and coherency root) once layer 0 is done; all land in
        // shared memory while the layers run.  After the output layer the
        // warps read its accumulator, hand the MMA warp the next tile's
        // features, and then scale and store this tile's WA.
        int tile = blockIdx.x;
        if (tile < n_tiles) {
            bool valid;
            int b, s;
            row_of(tile, valid, b, s);
            features(valid, b, valid ? lt.azza[(long long)t * lt.pitch + s] : make_float2(0.f, 0.f));
        }
        for (; tile < n_tiles && ok; tile += gridDim.x) {
            const int next = tile + gridDim.x;
            bool valid;
            int b, s;
            row_of(tile, valid, b, s);
            {
                bool nvalid = false;
                int nb = 0, ns = 0;
                if (next < n_tiles) row_of(next, nvalid, nb, ns);
                if (nvalid) cp_async<8>(my_azza, lt.azza + (long long)t * lt.pitch + ns);
            }
            const bool wa_row = h == 0 && valid;
            const int src = wa_row ? lt.idx[(long long)t * lt.pitch + s] : 0;
            // ---- hidden layers: accumulator -> bias, ReLU -> BF16 activations
            for (int l = 0; l < D; ++l) {
                if (!wait_bounded_spin(dfull, (uint32_t)(nd++) & 1u, abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                if (l == 0 && wa_row) {  // the source index has landed by now
                    cp_async<4>(smem_u32(&g_alpha[row]), m.half_alpha + src);
                    if (m.pol_m) cp_async<16>(smem_u32(&g_m[row]), m.pol_m + src);
                    else cp_async<4>(smem_u32(&g_m[row]), m.sqrt_flux + src);
                }
                if (l == 0) cp_async_commit();
                const float* bias = sbias + l * 256;
                // this warp's H / 2 columns, two 16-column TMEM loads in flight at a time
                auto drain = [&](const uint32_t (&a32)[16], int c0) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float4 b0 = *reinterpret_cast<const float4*>(bias + c0 + 8 * j);
                        const float4 b1 = *reinterpret_cast<const float4*>(bias + c0 + 8 * j + 4);
                        st_shared_v4(a_chunk(ab, r_loc, c0 + 8 * j),
                                     relu_bf16x2(__uint_as_float(a32[8 * j]) + b0.x, __uint_as_float(a32[8 * j + 1]) + b0.y),
                                     relu_bf16x2(__uint_as_float(a32[8 * j + 2]) + b0.z, __uint_as_float(a32[8 * j + 3]) + b0.w),
                                     relu_bf16x2(__uint_as_float(a32[8 * j + 4]) + b1.x, __uint_as_float(a32[8 * j + 5]) + b1.y),
                                     relu_bf16x2(__uint_as_float(a32[8 * j + 6]) + b1.z, __uint_as_float(a32[8 * j + 7]) + b1.w));
                    }
                };
                for (int c00 = h * (H / 2); c00 < (h + 1) * (H / 2); c00 += 32) {
                    uint32_t acc[2][16];
                    tmem_ld16(trow + c00, acc[0]);
                    tmem_ld16(trow + c00 + 16, acc[1]);
                    tmem_wait_ld16(acc[0]);
                    keep_after_wait16(acc[1]);
                    drain(acc[0], c00);
                    drain(acc[1], c00 + 16);
                }
                tc_fence_before();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(afull);
            }
            if (!ok) break;
            // ---- output layer: accumulator -> registers, then the next tile's
            // features (the accumulator columns are free again), then WA
            if (!wait_bounded_spin(dfull, (uint32_t)(nd++) & 1u, abort_flag, err)) { ok = false; break; }
            tc_fence_after();
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
            if (next < n_tiles) {
                bool nvalid;
                int nb, ns;
                row_of(next, nvalid, nb, ns);
                features(nvalid, nb, nvalid ? g_azza[threadIdx.x - 64] : make_float2(0.f, 0.f));
            }
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
                                wb[(long long)c * wa_pitch] = v;
                                mx = fmaxf(mx, hypotf(v.x, v.y));
                            }
                    } else {  // two axes per feed: z = A M (eq. "fullz")
#pragma unroll
                        for (int c = 0; c < 4; c += 2)
                            if (c + 1 < ncomp) {
                                float2 z0, z1;
                                apply_sky_sqrt(make_float2(y[2 * c], y[2 * c + 1]),
                                               make_float2(y[2 * c + 2], y[2 * c + 3]), gm, spec, z0, z1);
                                wb[(long long)c * wa_pitch] = z0;
                                wb[(long long)(c + 1) * wa_pitch] = z1;
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

}  // namespace

bool mlp_tc_supported(int F, int E, int H, int depth, int d0p, int n_out) {
    return (H == 128 || H == 256) && depth >= 1 && depth <= MAXL && d0p <= 256 && d0p % 16 == 0 && F % 8 == 0 &&
           E % 8 == 0 && n_out <= 8 && 2 * F + E <= d0p && F <= MAXF && get_encode() != nullptr;
}

cudaError_t mlp_tc_init() {
    return cudaFuncSetAttribute(k_mlp_wa, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t launch_mlp_wa_tc(const MlpTcArgs& a, const Model& m, LiveTables lt, int t, int K, float nu,
                             float ln_ratio, float2* wa_slot, long long wa_pitch, float* amax, int* d_err, int n_sms,
                             cudaStream_t st, long long* launches) {
    if (K <= 0 || a.n_beam <= 0) return cudaSuccess;
    if (!mlp_tc_supported(a.F, a.E, a.H, a.depth, a.d0p, a.n_out)) return cudaErrorInvalidValue;
    Maps maps{};
    for (int l = 0; l <= a.depth; ++l) {
        const int kin = l == 0 ? a.d0p : a.H;
        const int rows = l == a.depth ? 8 : a.H;
        const int box_rows = rows;
        if (!make_wmap(&maps.w[l], a.pb + a.off_w[l], kin, rows, box_rows)) return cudaErrorInvalidValue;
    }
    Net net{};
    net.F = a.F; net.E = a.E; net.H = a.H; net.depth = a.depth; net.d0p = a.d0p; net.n_beam = a.n_beam;
    net.n_out = a.n_out;
    net.nu_mid = a.nu_mid; net.nu_half = a.nu_half;
    net.p = a.p;
    for (int l = 0; l <= a.depth; ++l) net.off_b[l] = a.off_b[l];
    net.off_emb = a.off_emb;
    net.Bf = a.Bf;
    const long long R = (long long)a.n_beam * K;
    const int n_tiles = (int)((R + TM - 1) / TM);
    const int grid = std::max(1, std::min(n_sms, n_tiles));
    k_mlp_wa<<<grid, THREADS, SMEM_BYTES, st>>>(maps, net, m, lt, t, K, nu, ln_ratio, wa_slot, wa_pitch, amax, d_err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
