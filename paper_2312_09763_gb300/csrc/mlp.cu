// mlp.cu -- learned beam: a Fourier-feature MLP (antenna, az, za, nu) ->
// beam components, trained on the GPU against the gridded beam's own Keys
// interpolation, and evaluated in place of that interpolation.
//
// The paper's beams are interpolated from a grid (Sec. 2.4) and it notes that
// per-antenna beams make that step "highly non-negligible" (Sec. 3.1); the
// surrogate replaces n_ant gridded beams (n_ant x 4 x n_nu x n_za x n_az
// values) by one network of ~2.4e5 weights plus a 16-value embedding per
// antenna.  Definitions (shared with the test oracle only through this text):
//   x = (az / 2 pi, za / (pi/2), (nu - nu_mid) / nu_half)
//   f = [sin(2 pi B x), cos(2 pi B x), e_a]  (B: F x 3, az column integer)
//   h_l = relu(W_l h_{l-1} + b_l), y = W_out h_L + b_out;  MSE loss; Adam.
// Matrix products run on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation); master weights and Adam state are FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace mv {

typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------------------ GEMM
enum Epi : int { EPI_F32 = 0, EPI_BIAS_RELU_BF16 = 1, EPI_BIAS_F32 = 2, EPI_MASK_BF16 = 3, EPI_BF16 = 4, EPI_F32_ADD = 5 };

constexpr int GM = 128, GN = 128, GK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Load a GM x GK (or GN x GK) tile into shared memory laid out [row][k].
// kmajor: source stored [rows][K] with leading dimension ld (k contiguous);
// otherwise stored [K][rows] (row index contiguous).  Rows >= R or k >= K are
// zero.  K and ld are multiples of 8.
template <bool KMAJOR>
__device__ __forceinline__ void load_tile(bf16 (*S)[GK + GPAD], const bf16* __restrict__ src, int ld, int r0, int R,
                                          int k0, int K) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int idx = tid + q * 256;
        if (KMAJOR) {
            const int row = idx >> 2, ch = (idx & 3) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + row < R && k0 + ch < K) v = *reinterpret_cast<const uint4*>(src + (long long)(r0 + row) * ld + k0 + ch);
            *reinterpret_cast<uint4*>(&S[row][ch]) = v;
        } else {
            const int kr = idx >> 4, mc = (idx & 15) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k0 + kr < K && r0 + mc < R) {
                if (r0 + mc + 8 <= R) {
                    v = *reinterpret_cast<const uint4*>(src + (long long)(k0 + kr) * ld + r0 + mc);
                } else {
                    bf16 tmp[8];
                    for (int j = 0; j < 8; ++j)
                        tmp[j] = r0 + mc + j < R ? src[(long long)(k0 + kr) * ld + r0 + mc + j] : __float2bfloat16(0.f);
                    v = *reinterpret_cast<uint4*>(tmp);
                }
            }
            const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) S[mc + j][kr] = e[j];
        }
    }
}

// C[M][N] = op(A)[M][K] op(B)[K][N] with a fused epilogue (see Epi).
// A_KM: A stored [M][K], else [K][M].  B_KM: B stored [N][K], else [K][N].
// blockIdx.z takes the k-range [z kc, (z + 1) kc); with EPI_F32_ADD the
// partial products are added into C (which the caller zeroes).
template <bool A_KM, bool B_KM>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, int K, const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb, void* C, int ldc,
       int epi, const float* __restrict__ bias, const bf16* __restrict__ mask, int ldm, int kc) {
    __shared__ __align__(16) bf16 As[GM][GK + GPAD];
    __shared__ __align__(16) bf16 Bs[GN][GK + GPAD];
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps: 64 x 32 each
    const int g = lane >> 2, t = lane & 3;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    for (int k0 = kb; k0 < ke; k0 += GK) {
        load_tile<A_KM>(As, A, lda, m0, M, k0, ke);
        load_tile<B_KM>(Bs, B, ldb, n0, N, k0, ke);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk += 16) {
            uint32_t af[4][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wm * 64 + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn * 32 + j * 8 + g;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * t]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 64 + i * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * t + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                const long long o = (long long)m * ldc + n;
                if (epi == EPI_F32) {
                    static_cast<float*>(C)[o] = v;
                } else if (epi == EPI_F32_ADD) {
                    atomicAdd(static_cast<float*>(C) + o, v);
                } else if (epi == EPI_BIAS_F32) {
                    static_cast<float*>(C)[o] = v + bias[n];
                } else if (epi == EPI_BIAS_RELU_BF16) {
                    static_cast<bf16*>(C)[o] = __float2bfloat16(fmaxf(v + bias[n], 0.f));
                } else if (epi == EPI_BF16) {
                    static_cast<bf16*>(C)[o] = __float2bfloat16(v);
                } else {
                    const float mk = __bfloat162float(mask[(long long)m * ldm + n]) > 0.f ? 1.f : 0.f;
                    static_cast<bf16*>(C)[o] = __float2bfloat16(v * mk);
                }
            }
}

cudaError_t gemm(bool a_km, bool b_km, int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, void* C,
                 int ldc, int epi, const float* bias, const bf16* mask, int ldm, cudaStream_t st, long long* L) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM, 1);
    int kc = (K + GK - 1) / GK * GK;
    if (epi == EPI_F32_ADD) {
        // split the (long) k axis so that the grid fills the GPU
        const int tiles = grid.x * grid.y;
        const int ks = std::max(1, std::min((K + 127) / 128, 600 / std::max(tiles, 1)));
        kc = ((K + ks - 1) / ks + GK - 1) / GK * GK;
        grid.z = (K + kc - 1) / kc;
    }
    if (a_km && b_km)
        k_gemm<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask, ldm, kc);
    else if (a_km)
        k_gemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask, ldm, kc);
    else if (b_km)
        k_gemm<false, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask, ldm, kc);
    else
        k_gemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask, ldm, kc);
    ++*L;
    return cudaGetLastError();
}

// ------------------------------------------------------- small kernels
struct Dims {
    int F, E, H, depth, n_out, n_ant;
    int d0, d0p;  // feature width 2F + E, padded to a multiple of 32
    float nu_mid, nu_half;
};

// Fourier features + embedding: X0[m][0..d0p) in BF16 (zero padding).
__global__ void k_features(Dims d, const float* __restrict__ Bf, const float* __restrict__ emb, int M,
                           const int* __restrict__ ant, const float* __restrict__ az, const float* __restrict__ za,
                           const float* __restrict__ nu, bf16* __restrict__ X0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * d.d0p) return;
    const int m = (int)(i / d.d0p), j = (int)(i % d.d0p);
    float v = 0.f;
    if (j < 2 * d.F) {
        const int f = j % d.F;
        const float x0 = az[m] * 0.15915494309189535f;           // az / 2 pi
        const float x1 = za[m] * 0.63661977236758134f;           // za / (pi / 2)
        const float x2 = (nu[m] - d.nu_mid) / d.nu_half;
        float ph = Bf[3 * f] * x0 + Bf[3 * f + 1] * x1 + Bf[3 * f + 2] * x2;  // turns
        ph -= rintf(ph);
        float s, c;
        sincospif(2.f * ph, &s, &c);
        v = j < d.F ? s : c;
    } else if (j < d.d0) {
        v = emb[(long long)ant[m] * d.E + (j - 2 * d.F)];
    }
    X0[i] = __float2bfloat16(v);
}

// dY = 2 (y - t) / (M n_out) (BF16, padded outputs zero) and sum of squares.
__global__ void k_loss(int M, int n_out, const float* __restrict__ Y, const float* __restrict__ T,
                       bf16* __restrict__ dY, double* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float r2 = 0.f;
    if (i < M * 8) {
        const int m = i >> 3, o = i & 7;
        float g = 0.f;
        if (o < n_out) {
            const float r = Y[i] - T[(long long)m * n_out + o];
            r2 = r * r;
            g = 2.f * r / (float)((long long)M * n_out);
        }
        dY[i] = __float2bfloat16(g);
    }
    for (int off = 16; off > 0; off >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)r2);
}

// db[n] = sum_m dZ[m][n] (fixed order: one thread per column, rows in sequence
// over a strided split, then a fixed tree in shared memory).
__global__ void k_colsum(int M, int N, const bf16* __restrict__ dZ, int ld, float* __restrict__ db) {
    __shared__ float part[8][32];
    const int n = blockIdx.x * 32 + (threadIdx.x & 31), r = threadIdx.x >> 5;
    float s = 0.f;
    if (n < N)
        for (int m = r; m < M; m += 8) s += __bfloat162float(dZ[(long long)m * ld + n]);
    part[r][threadIdx.x & 31] = s;
    __syncthreads();
    if (r == 0 && n < N) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += part[q][threadIdx.x & 31];
        db[n] = t;
    }
}

// Embedding gradient: columns [2F, 2F + E) of dX0, summed per antenna.
__global__ void k_emb_grad(Dims d, int M, const int* __restrict__ ant, const bf16* __restrict__ dX0,
                           float* __restrict__ gemb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * d.E) return;
    const int m = i / d.E, e = i % d.E;
    atomicAdd(&gemb[(long long)ant[m] * d.E + e], __bfloat162float(dX0[(long long)m * d.d0p + 2 * d.F + e]));
}

// Adam on one parameter array; writes the BF16 copy used by the products.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ pb, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
}

__global__ void k_to_bf16(long long n, const float* __restrict__ p, bf16* __restrict__ q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16(p[i]);
}

// ----------------------------------------------------- training samples
// splitmix64 (Steele, Lea and Flood 2014): a counter-based stream of 64-bit
// values; uniform doubles take its top 53 bits.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long ctr) {
    return (double)(splitmix64(seed ^ splitmix64(ctr)) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ float keys_w(float x) {
    const float t = fabsf(x);
    if (t <= 1.f) return (1.5f * t - 2.5f) * t * t + 1.f;
    if (t < 2.f) return ((-0.5f * t + 2.5f) * t - 4.f) * t + 2.f;
    return 0.f;
}

// Keys-cubic interpolation of component `comp` of beam `b` of the raw grid at
// (az, za) and fractional frequency node u (Sec. 2.4; pole and az wrap as in
// the beam step of the simulator).
__device__ float2 grid_value(const Model& m, const float2* __restrict__ grid, int b, int comp, float az, float za,
                             float u) {
    const long long plane = (long long)m.n_za * m.n_az;
    const float2* G = grid + ((long long)b * m.n_feed * m.n_ax + comp) * m.n_nu * plane;
    const float fu = floorf(u), tu = u - fu;
    const int f0 = (int)fu - 1;
    const float wf[4] = {keys_w(tu + 1.f), keys_w(tu), keys_w(1.f - tu), keys_w(2.f - tu)};
    const float uz = za / m.dza, ua = az / m.daz;
    const float fz = floorf(uz), fa = floorf(ua);
    const float tz = uz - fz, ta = ua - fa;
    const int z0 = (int)fz - 1, a0 = (int)fa - 1;
    const float wz[4] = {keys_w(tz + 1.f), keys_w(tz), keys_w(1.f - tz), keys_w(2.f - tz)};
    const float wa[4] = {keys_w(ta + 1.f), keys_w(ta), keys_w(1.f - ta), keys_w(2.f - ta)};
    const float pole_sign = m.n_ax == 2 ? -1.f : 1.f;
    float re = 0.f, im = 0.f;
    for (int r = 0; r < 4; ++r) {
        int row = z0 + r, sh = 0;
        float sg = 1.f;
        if (row < 0) { row = -row; sh = m.n_az / 2; sg = pole_sign; }
        if (row > m.n_za - 1) row = m.n_za - 1;
        for (int q = 0; q < 4; ++q) {
            int col = (a0 + q + sh) % m.n_az;
            if (col < 0) col += m.n_az;
            const float w2 = wz[r] * wa[q] * sg;
            for (int j = 0; j < 4; ++j) {
                const float2 v = G[(long long)(f0 + j) * plane + (long long)row * m.n_az + col];
                re = fmaf(w2 * wf[j], v.x, re);
                im = fmaf(w2 * wf[j], v.y, im);
            }
        }
    }
    return make_float2(re, im);
}

// Draw M training samples (antenna, az, za, nu) uniformly (nu inside the
// grid's cubic margin) and their targets from the gridded beams.
__global__ void k_sample(Model m, const float2* __restrict__ grid, double nu0, double dnu, double nu_lo,
                         double nu_hi, unsigned long long seed, unsigned long long step, int M, int n_out,
                         int* __restrict__ ant, float* __restrict__ az, float* __restrict__ za, float* __restrict__ nu,
                         float* __restrict__ T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const unsigned long long base = (step * (unsigned long long)M + i) * 4ull;
    const int a = min(m.n_beam - 1, (int)(uniform01(seed, base) * m.n_beam));
    const double vaz = uniform01(seed, base + 1) * 2.0 * kPi;
    const double vza = uniform01(seed, base + 2) * 0.5 * kPi;
    const double vnu = nu_lo + uniform01(seed, base + 3) * (nu_hi - nu_lo);
    ant[i] = a;
    az[i] = (float)vaz;
    za[i] = (float)vza;
    nu[i] = (float)vnu;
    const float u = (float)((vnu - nu0) / dnu);
    const int ncomp = m.n_feed * m.n_ax;
    for (int c = 0; c < ncomp && 2 * c < n_out; ++c) {
        const float2 v = grid_value(m, grid, a, c, (float)vaz, (float)vza, u);
        T[(long long)i * n_out + 2 * c] = v.x;
        T[(long long)i * n_out + 2 * c + 1] = v.y;
    }
}

// Rows (beta, s) of one instance for the surrogate: antenna beta and the live
// source s's (az, za) at the instance's frequency.
__global__ void k_rows(int n_ant, int K, long long r0, int R, int t, float nu, LiveTables lt, int* __restrict__ ant,
                       float* __restrict__ az, float* __restrict__ za, float* __restrict__ vnu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    const long long r = r0 + i;
    const int b = (int)(r / K), s = (int)(r % K);
    const float2 p = lt.azza[(long long)t * lt.pitch + s];
    ant[i] = b;
    az[i] = p.x;
    za[i] = p.y;
    vnu[i] = nu;
}

// WA[slot][beta][comp][s] = sqrt(I_s(nu)) * (y[2 comp], y[2 comp + 1]).
__global__ void k_wa_rows(Model m, int K, long long r0, int R, int t, float ln_ratio, LiveTables lt,
                          const float* __restrict__ Y, int ncomp, float2* __restrict__ wa_slot, long long wa_pitch,
                          float* __restrict__ amax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float mx = 0.f;
    if (i < R) {
        const long long r = r0 + i;
        const int b = (int)(r / K), s = (int)(r % K);
        const int src = lt.idx[(long long)t * lt.pitch + s];
        const float spec = expf(m.half_alpha[src] * ln_ratio);
        if (!m.pol_m) {
            const float w = m.sqrt_flux[src] * spec;
            for (int c = 0; c < ncomp; ++c) {
                const float2 v = make_float2(w * Y[(long long)i * 8 + 2 * c], w * Y[(long long)i * 8 + 2 * c + 1]);
                wa_slot[((long long)b * ncomp + c) * wa_pitch + s] = v;
                mx = fmaxf(mx, hypotf(v.x, v.y));
            }
        } else {  // two axes per feed: z = A M (eq. "fullz")
            const float4 M = m.pol_m[src];
            for (int c = 0; c + 1 < ncomp; c += 2) {
                const float* y = Y + (long long)i * 8 + 2 * c;
                float2 z0, z1;
                apply_sky_sqrt(make_float2(y[0], y[1]), make_float2(y[2], y[3]), M, spec, z0, z1);
                wa_slot[((long long)b * ncomp + c) * wa_pitch + s] = z0;
                wa_slot[((long long)b * ncomp + c + 1) * wa_pitch + s] = z1;
                mx = fmaxf(mx, fmaxf(hypotf(z0.x, z0.y), hypotf(z1.x, z1.y)));
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(reinterpret_cast<int*>(amax), __float_as_int(mx));
}

unsigned gridsz(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------- state
struct Surrogate {
    Dims d{};
    // parameter vector layout (FP32 master / BF16 copy / Adam m, v / grads)
    std::vector<long long> off_w, off_b;  // per layer (depth hidden + output)
    long long off_emb = 0, n_par = 0;
    float* p = nullptr;
    float* g = nullptr;
    float* am = nullptr;
    float* av = nullptr;
    bf16* pb = nullptr;
    float* Bf = nullptr;  // Fourier matrix [F][3]
    std::vector<float> hB;
    long long adam_k = 0;
    // work buffers for up to `cap` rows
    long long cap = 0;
    int *ant = nullptr;
    float *az = nullptr, *za = nullptr, *nu = nullptr, *T = nullptr, *Y = nullptr;
    bf16 *X0 = nullptr, *dX0 = nullptr, *dY = nullptr;
    std::vector<bf16*> Hs;  // hidden activations (training keeps all layers)
    bf16 *dZa = nullptr, *dZb = nullptr;
    double* loss = nullptr;
};

namespace {

void sfree(void* p) {
    if (p) cudaFree(p);
}

cudaError_t ensure_rows(Surrogate* S, long long rows) {
    if (rows <= S->cap) return cudaSuccess;
    sfree(S->ant); sfree(S->az); sfree(S->za); sfree(S->nu); sfree(S->T); sfree(S->Y);
    sfree(S->X0); sfree(S->dX0); sfree(S->dY); sfree(S->dZa); sfree(S->dZb);
    for (auto* h : S->Hs) sfree(h);
    S->Hs.assign(S->d.depth, nullptr);
    cudaError_t e = cudaSuccess;
    auto A = [&](void** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(q, bytes);
    };
    const Dims& d = S->d;
    A((void**)&S->ant, sizeof(int) * rows);
    A((void**)&S->az, sizeof(float) * rows);
    A((void**)&S->za, sizeof(float) * rows);
    A((void**)&S->nu, sizeof(float) * rows);
    A((void**)&S->T, sizeof(float) * rows * 8);
    A((void**)&S->Y, sizeof(float) * rows * 8);
    A((void**)&S->X0, sizeof(bf16) * rows * d.d0p);
    A((void**)&S->dX0, sizeof(bf16) * rows * d.d0p);
    A((void**)&S->dY, sizeof(bf16) * rows * 8);
    A((void**)&S->dZa, sizeof(bf16) * rows * d.H);
    A((void**)&S->dZb, sizeof(bf16) * rows * d.H);
    for (int l = 0; l < d.depth; ++l) A((void**)&S->Hs[l], sizeof(bf16) * rows * d.H);
    if (e == cudaSuccess) S->cap = rows;
    return e;
}

// Forward pass of `rows` rows whose features are in X0: hidden layers into
// Hs[l] (all kept for training) and the FP32 output into Y [rows][8].
cudaError_t forward(Surrogate* S, int rows, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    cudaError_t e = cudaSuccess;
    const bf16* in = S->X0;
    int kin = d.d0p;
    for (int l = 0; l < d.depth && e == cudaSuccess; ++l) {
        e = gemm(true, true, rows, d.H, kin, in, kin, S->pb + S->off_w[l], kin, S->Hs[l], d.H, EPI_BIAS_RELU_BF16,
                 S->p + S->off_b[l], nullptr, 0, st, L);
        in = S->Hs[l];
        kin = d.H;
    }
    if (e == cudaSuccess)
        e = gemm(true, true, rows, 8, d.H, in, d.H, S->pb + S->off_w[d.depth], d.H, S->Y, 8, EPI_BIAS_F32,
                 S->p + S->off_b[d.depth], nullptr, 0, st, L);
    return e;
}

// Backward pass for the batch in X0 / Hs / dY: all gradients into S->g.
cudaError_t backward(Surrogate* S, int rows, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    // weight and embedding gradients accumulate (split over the batch): zero all
    cudaError_t e = cudaMemsetAsync(S->g, 0, sizeof(float) * (size_t)S->n_par, st);
    // output layer: dW_out = dY^T H_L, db_out = sum dY, dH_L = (dY W_out) * (H_L > 0)
    const int D = d.depth;
    bf16* dz = S->dZa;
    bf16* dz_next = S->dZb;
    if (e == cudaSuccess)
        e = gemm(false, false, 8, d.H, rows, S->dY, 8, S->Hs[D - 1], d.H, S->g + S->off_w[D], d.H, EPI_F32_ADD,
                 nullptr, nullptr, 0, st, L);
    if (e == cudaSuccess) {
        k_colsum<<<gridsz(8, 32), 256, 0, st>>>(rows, 8, S->dY, 8, S->g + S->off_b[D]);
        ++*L;
        e = gemm(true, false, rows, d.H, 8, S->dY, 8, S->pb + S->off_w[D], d.H, dz, d.H, EPI_MASK_BF16, nullptr,
                 S->Hs[D - 1], d.H, st, L);
    }
    for (int l = D - 1; l >= 0 && e == cudaSuccess; --l) {
        const bf16* in = l == 0 ? S->X0 : S->Hs[l - 1];
        const int kin = l == 0 ? d.d0p : d.H;
        // dW_l = dZ^T in, db_l = sum dZ
        e = gemm(false, false, d.H, kin, rows, dz, d.H, in, kin, S->g + S->off_w[l], kin, EPI_F32_ADD, nullptr, nullptr,
                 0, st, L);
        if (e != cudaSuccess) break;
        k_colsum<<<gridsz(d.H, 32), 256, 0, st>>>(rows, d.H, dz, d.H, S->g + S->off_b[l]);
        ++*L;
        if (l > 0) {
            e = gemm(true, false, rows, d.H, d.H, dz, d.H, S->pb + S->off_w[l], d.H, dz_next, d.H, EPI_MASK_BF16,
                     nullptr, S->Hs[l - 1], d.H, st, L);
            std::swap(dz, dz_next);
        } else {
            // features: only the embedding columns need a gradient
            e = gemm(true, false, rows, d.d0p, d.H, dz, d.H, S->pb + S->off_w[0], d.d0p, S->dX0, d.d0p, EPI_BF16,
                     nullptr, nullptr, 0, st, L);
        }
    }
    if (e == cudaSuccess) {
        k_emb_grad<<<gridsz((long long)rows * d.E, 256), 256, 0, st>>>(d, rows, S->ant, S->dX0, S->g + S->off_emb);
        ++*L;
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

Surrogate* surrogate_create(int F, int E, int H, int depth, int n_out, int n_ant, float s_az, float s_za, float s_nu,
                            unsigned long long seed, double nu_mid, double nu_half, cudaError_t* err) {
    Surrogate* S = new Surrogate();
    Dims& d = S->d;
    d.F = F; d.E = E; d.H = H; d.depth = depth; d.n_out = n_out; d.n_ant = n_ant;
    d.d0 = 2 * F + E;
    d.d0p = (d.d0 + 31) / 32 * 32;
    d.nu_mid = (float)nu_mid;
    d.nu_half = (float)nu_half;
    long long o = 0;
    for (int l = 0; l <= depth; ++l) {
        const int kin = l == 0 ? d.d0p : H;
        const int nout = l == depth ? 8 : H;
        S->off_w.push_back(o);
        o += (long long)nout * kin;
        S->off_b.push_back(o);
        o += nout;
        o = (o + 7) / 8 * 8;  // keep every array 16-byte aligned
    }
    S->off_emb = o;
    o += (long long)n_ant * E;
    S->n_par = o;
    // host initialisation (He-normal weights, zero biases, small embeddings)
    std::vector<float> hp(o, 0.f);
    unsigned long long state = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        state += 0x9E3779B97F4A7C15ull;
        unsigned long long x = state;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        return ((x ^ (x >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() {  // Box-Muller
        const double u1 = std::max(next(), 1e-300), u2 = next();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * kPi * u2);
    };
    for (int l = 0; l <= depth; ++l) {
        const int kin = l == 0 ? d.d0 : H, kinp = l == 0 ? d.d0p : H;
        const int nout = l == depth ? n_out : H;
        const double sd = std::sqrt(2.0 / kin) * (l == depth ? 0.5 : 1.0);
        for (int r = 0; r < nout; ++r)
            for (int c = 0; c < kin; ++c) hp[S->off_w[l] + (long long)r * kinp + c] = (float)(sd * normal());
    }
    for (long long i = 0; i < (long long)n_ant * E; ++i) hp[S->off_emb + i] = (float)(0.1 * normal());
    S->hB.resize(3 * F);
    for (int f = 0; f < F; ++f) {
        S->hB[3 * f] = (float)std::nearbyint(s_az * normal());
        S->hB[3 * f + 1] = (float)(s_za * normal());
        S->hB[3 * f + 2] = (float)(s_nu * normal());
    }
    cudaError_t e = cudaMalloc(&S->p, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->g, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->am, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->av, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->pb, sizeof(bf16) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->Bf, sizeof(float) * 3 * F);
    if (e == cudaSuccess) e = cudaMemcpy(S->p, hp.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S->Bf, S->hB.data(), sizeof(float) * 3 * F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(S->g, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(S->am, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(S->av, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMalloc(&S->loss, sizeof(double));
    if (e == cudaSuccess) {
        k_to_bf16<<<gridsz(o, 256), 256>>>(o, S->p, S->pb);
        e = cudaDeviceSynchronize();
    }
    *err = e;
    if (e != cudaSuccess) {
        surrogate_destroy(S);
        return nullptr;
    }
    return S;
}

void surrogate_destroy(Surrogate* S) {
    if (!S) return;
    cudaDeviceSynchronize();
    for (void* q : {(void*)S->p, (void*)S->g, (void*)S->am, (void*)S->av, (void*)S->pb, (void*)S->Bf, (void*)S->ant,
                    (void*)S->az, (void*)S->za, (void*)S->nu, (void*)S->T, (void*)S->Y, (void*)S->X0, (void*)S->dX0,
                    (void*)S->dY, (void*)S->dZa, (void*)S->dZb, (void*)S->loss})
        sfree(q);
    for (auto* h : S->Hs) sfree(h);
    delete S;
}

long long surrogate_param_count(const Surrogate* S) { return S->n_par; }
int surrogate_fourier(const Surrogate* S, float* out) {
    std::memcpy(out, S->hB.data(), sizeof(float) * S->hB.size());
    return (int)S->hB.size();
}
void surrogate_layout(const Surrogate* S, long long* off_w, long long* off_b, long long* off_emb, int* d0p) {
    for (int l = 0; l <= S->d.depth; ++l) {
        off_w[l] = S->off_w[l];
        off_b[l] = S->off_b[l];
    }
    *off_emb = S->off_emb;
    *d0p = S->d.d0p;
}

cudaError_t surrogate_get_params(const Surrogate* S, float* host) {
    return cudaMemcpy(host, S->p, sizeof(float) * S->n_par, cudaMemcpyDeviceToHost);
}

cudaError_t surrogate_set_params(Surrogate* S, const float* host) {
    cudaError_t e = cudaMemcpy(S->p, host, sizeof(float) * S->n_par, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_to_bf16<<<gridsz(S->n_par, 256), 256>>>(S->n_par, S->p, S->pb);
        e = cudaDeviceSynchronize();
    }
    S->adam_k = 0;
    if (e == cudaSuccess) e = cudaMemset(S->am, 0, sizeof(float) * S->n_par);
    if (e == cudaSuccess) e = cudaMemset(S->av, 0, sizeof(float) * S->n_par);
    return e;
}

// Forward + backward on caller-given samples (host arrays), gradients to host
// (the check of the GPU gradients against the FP64 oracle).
cudaError_t surrogate_grad(Surrogate* S, int n, const int* ant, const float* az, const float* za, const float* nu,
                           const float* T, float* grads_host, double* loss, cudaStream_t st) {
    cudaError_t e = ensure_rows(S, n);
    long long L = 0;
    const Dims& d = S->d;
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->ant, ant, sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->az, az, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->za, za, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->nu, nu, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->T, T, sizeof(float) * n * d.n_out, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_features<<<gridsz((long long)n * d.d0p, 256), 256, 0, st>>>(d, S->Bf, S->p + S->off_emb, n, S->ant, S->az, S->za,
                                                                    S->nu, S->X0);
    e = forward(S, n, st, &L);
    if (e == cudaSuccess) {
        k_loss<<<gridsz((long long)n * 8, 256), 256, 0, st>>>(n, d.n_out, S->Y, S->T, S->dY, S->loss);
        e = backward(S, n, st, &L);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(grads_host, S->g, sizeof(float) * S->n_par, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, S->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) *loss /= (double)n * d.n_out;
    return e;
}

// Evaluate the network at caller-given points (host arrays): out [n][n_out].
cudaError_t surrogate_eval(Surrogate* S, int n, const int* ant, const float* az, const float* za, const float* nu,
                           float* out_host, cudaStream_t st) {
    cudaError_t e = ensure_rows(S, n);
    long long L = 0;
    const Dims& d = S->d;
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->ant, ant, sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->az, az, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->za, za, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->nu, nu, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_features<<<gridsz((long long)n * d.d0p, 256), 256, 0, st>>>(d, S->Bf, S->p + S->off_emb, n, S->ant, S->az, S->za,
                                                                    S->nu, S->X0);
    e = forward(S, n, st, &L);
    if (e != cudaSuccess) return e;
    std::vector<float> y((size_t)n * 8);
    e = cudaMemcpyAsync(y.data(), S->Y, sizeof(float) * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int i = 0; i < n; ++i)
        for (int o = 0; o < d.n_out; ++o) out_host[(size_t)i * d.n_out + o] = y[(size_t)i * 8 + o];
    return e;
}

// Train for `steps` Adam steps of `batch` samples drawn from the gridded beam
// (cosine learning-rate schedule from lr0 to lr1).  Reports the loss of the
// first and of the last step.
cudaError_t surrogate_train(Surrogate* S, const Model& m, const float2* grid, double nu0, double dnu, int steps,
                            int batch, float lr0, float lr1, unsigned long long seed, cudaStream_t st,
                            double* loss_first, double* loss_last, long long* L) {
    cudaError_t e = ensure_rows(S, batch);
    if (e != cudaSuccess) return e;
    const Dims& d = S->d;
    const double nu_lo = nu0 + 1.0 * dnu, nu_hi = nu0 + (m.n_nu - 3) * dnu * 0.999999;
    for (int it = 0; it < steps && e == cudaSuccess; ++it) {
        if (it == 0 || it == steps - 1) e = cudaMemsetAsync(S->loss, 0, sizeof(double), st);
        k_sample<<<gridsz(batch, 128), 128, 0, st>>>(m, grid, nu0, dnu, nu_lo, nu_hi, seed, (unsigned long long)it,
                                                      batch, d.n_out, S->ant, S->az, S->za, S->nu, S->T);
        k_features<<<gridsz((long long)batch * d.d0p, 256), 256, 0, st>>>(d, S->Bf, S->p + S->off_emb, batch, S->ant,
                                                                            S->az, S->za, S->nu, S->X0);
        *L += 2;
        e = forward(S, batch, st, L);
        if (e != cudaSuccess) break;
        k_loss<<<gridsz((long long)batch * 8, 256), 256, 0, st>>>(batch, d.n_out, S->Y, S->T, S->dY, S->loss);
        ++*L;
        if (it == 0 || it == steps - 1) {
            double l = 0;
            e = cudaMemcpyAsync(&l, S->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            l /= (double)batch * d.n_out;
            if (it == 0) *loss_first = l;
            if (it == steps - 1) *loss_last = l;
        }
        e = backward(S, batch, st, L);
        if (e != cudaSuccess) break;
        const float lr = lr1 + 0.5f * (lr0 - lr1) * (1.f + cosf((float)kPi * it / std::max(1, steps - 1)));
        S->adam_k += 1;
        const float c1 = 1.f - powf(0.9f, (float)S->adam_k), c2 = 1.f - powf(0.999f, (float)S->adam_k);
        k_adam<<<gridsz(S->n_par, 256), 256, 0, st>>>(S->n_par, S->p, S->g, S->am, S->av, S->pb, lr, 0.9f, 0.999f,
                                                       1e-8f, c1, c2);
        ++*L;
        e = cudaGetLastError();
    }
    return e;
}

// Beam x sqrt(I) for every (antenna, live source) of instances inst0 ..
// inst0 + n_inst - 1 from the network, into WA slots (n_beam = n_ant layout).
cudaError_t surrogate_wa(Surrogate* S, const Model& m, const std::vector<Inst>& h_inst, int inst0, int n_inst,
                         const std::vector<int>& h_nlive, const std::vector<double>& h_nu, double nu_ref, LiveTables lt,
                         float2* wa, long long wa_pitch, float* amax, int* d_err, int n_sms, cudaStream_t st,
                         long long* L) {
    const Dims& d = S->d;
    const int ncomp = m.n_feed * m.n_ax;
    const long long chunk = 1 << 19;
    // the tensor-core forward pass (features, layers and WA in one launch per
    // instance) where the network shape allows, else the mma.sync GEMMs
    const bool tc = mlp_tc_supported(d.F, d.E, d.H, d.depth, d.d0p, d.n_out);
    MlpTcArgs ta{};
    if (tc) {
        ta.F = d.F; ta.E = d.E; ta.H = d.H; ta.depth = d.depth; ta.d0p = d.d0p; ta.n_beam = d.n_ant;
        ta.n_out = d.n_out; ta.nu_mid = d.nu_mid; ta.nu_half = d.nu_half;
        ta.p = S->p; ta.pb = S->pb; ta.off_emb = S->off_emb; ta.Bf = S->Bf;
        for (int l = 0; l <= d.depth; ++l) { ta.off_w[l] = S->off_w[l]; ta.off_b[l] = S->off_b[l]; }
    }
    cudaError_t e = tc ? cudaSuccess : ensure_rows(S, chunk);
    for (int j = 0; j < n_inst && e == cudaSuccess; ++j) {
        const Inst& in = h_inst[inst0 + j];
        const int K = h_nlive[in.t];
        const long long rows = (long long)d.n_ant * K;
        const float nu = (float)h_nu[in.c];
        const float lnr = (float)std::log(h_nu[in.c] / nu_ref);
        float2* wslot = wa + (long long)j * m.n_beam * ncomp * wa_pitch;
        if (tc) e = launch_mlp_wa_tc(ta, m, lt, in.t, K, nu, lnr, wslot, wa_pitch, amax + j, d_err, n_sms, st, L);
        for (long long r0 = 0; !tc && r0 < rows && e == cudaSuccess; r0 += chunk) {
            const int R = (int)std::min(chunk, rows - r0);
            k_rows<<<gridsz(R, 256), 256, 0, st>>>(d.n_ant, K, r0, R, in.t, nu, lt, S->ant, S->az, S->za, S->nu);
            k_features<<<gridsz((long long)R * d.d0p, 256), 256, 0, st>>>(d, S->Bf, S->p + S->off_emb, R, S->ant,
                                                                            S->az, S->za, S->nu, S->X0);
            *L += 2;
            e = forward(S, R, st, L);
            if (e != cudaSuccess) break;
            k_wa_rows<<<gridsz(R, 256), 256, 0, st>>>(m, K, r0, R, in.t, lnr, lt, S->Y, ncomp, wslot, wa_pitch,
                                                       amax + j);
            ++*L;
            e = cudaGetLastError();
        }
        // zeros past the live count (the Z build reads whole source pairs)
        if (e == cudaSuccess && K < wa_pitch)
            e = cudaMemset2DAsync(wslot + K, sizeof(float2) * wa_pitch, 0, sizeof(float2) * (wa_pitch - K),
                                  (size_t)m.n_beam * ncomp, st);
    }
    return e;
}

}  // namespace mv
