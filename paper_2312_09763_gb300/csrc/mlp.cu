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
// Every matrix product of a training step runs on the tcgen05 tensor cores
// (BF16 operands staged by TMA, FP32 accumulation in TMEM); master weights and
// Adam state are FP32.  A step is one fused launch for the row-local part
// (mlp_chain_tc.cu: features, forward, loss, input gradients, embedding
// gradient), one for every weight and bias gradient (mlp_wgrad_tc.cu: dW =
// dZ^T X with dZ and X read batch-major, the bias gradients as row sums of
// dZ^T from an extra MMA) and the optimiser step, while the next step's
// samples are drawn on a side stream (networks the fused launch does not
// cover run product by product, mlp_train_tc.cu); the input gradients read
// BF16 copies of W^T that the optimiser keeps.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"
#include "sample.cuh"

namespace mv {

typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------- small kernels
struct Dims {
    int F, E, H, depth, n_out, n_ant;
    int d0, d0p;  // feature width 2F + E, padded to a multiple of 32 (at least 64)
    float nu_mid, nu_half;
};

// Fourier features + embedding: X0[m][0..d0p) in BF16 (zero padding), and
// with X0T (may be NULL) the same values as columns, X0T[j][m] (ld ldt).  A
// block of 256 threads takes 64 rows: each (row, frequency) pair evaluates
// its sine and cosine once into a shared-memory tile, which is then written
// out as rows (and columns), coalesced.  Dynamic shared memory: 64 (d0p + 2)
// BF16 values.
constexpr int kFeatRows = 64;
__global__ void __launch_bounds__(256)
k_features(Dims d, const float* __restrict__ Bf, const float* __restrict__ emb, int M, const int* __restrict__ ant,
           const float* __restrict__ az, const float* __restrict__ za, const float* __restrict__ nu,
           bf16* __restrict__ X0, bf16* __restrict__ X0T, long long ldt) {
    extern __shared__ bf16 tile[];  // [kFeatRows][d0p + 2]
    const int ld = d.d0p + 2;
    const int m0 = blockIdx.x * kFeatRows;
    const int rl = threadIdx.x % kFeatRows, cg = threadIdx.x / kFeatRows;  // row, column group (4)
    const int m = m0 + rl;
    const bool valid = m < M;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    int a = 0;
    if (valid) {
        x0 = az[m] * 0.15915494309189535f;  // az / 2 pi
        x1 = za[m] * 0.63661977236758134f;  // za / (pi / 2)
        x2 = (nu[m] - d.nu_mid) / d.nu_half;
        a = ant[m];
    }
    for (int f = cg; f < d.F; f += 4) {
        float ph = Bf[3 * f] * x0 + Bf[3 * f + 1] * x1 + Bf[3 * f + 2] * x2;  // turns
        ph -= rintf(ph);
        float sv, cv;
        sincospif(2.f * ph, &sv, &cv);
        tile[rl * ld + f] = __float2bfloat16(valid ? sv : 0.f);
        tile[rl * ld + d.F + f] = __float2bfloat16(valid ? cv : 0.f);
    }
    for (int j = 2 * d.F + cg; j < d.d0p; j += 4)
        tile[rl * ld + j] = __float2bfloat16(valid && j < d.d0 ? emb[(long long)a * d.E + (j - 2 * d.F)] : 0.f);
    __syncthreads();
    // rows: consecutive threads along a row
    for (int q = threadIdx.x; q < kFeatRows * d.d0p; q += blockDim.x) {
        const int r = q / d.d0p, j = q % d.d0p;
        if (m0 + r < M) X0[(long long)(m0 + r) * d.d0p + j] = tile[r * ld + j];
    }
    if (X0T) {
        // columns: consecutive threads along m
        for (int q = threadIdx.x; q < kFeatRows * d.d0p; q += blockDim.x) {
            const int j = q / kFeatRows, r = q % kFeatRows;
            if (m0 + r < M) X0T[(long long)j * ldt + m0 + r] = tile[r * ld + j];
        }
    }
}

cudaError_t launch_features(const Dims& d, const float* Bf, const float* emb, int M, const int* ant, const float* az,
                            const float* za, const float* nu, bf16* X0, bf16* X0T, long long ldt, cudaStream_t st) {
    const size_t sm = sizeof(bf16) * kFeatRows * (size_t)(d.d0p + 2);
    k_features<<<(unsigned)((M + kFeatRows - 1) / kFeatRows), 256, sm, st>>>(d, Bf, emb, M, ant, az, za, nu, X0, X0T,
                                                                            ldt);
    return cudaGetLastError();
}

__global__ void k_to_bf16(long long n, const float* __restrict__ p, bf16* __restrict__ q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16(p[i]);
}

// The network's layers as the kernels below walk them: hidden layers, then
// the output layer.  The weight gradient of layer l is summed from `splits`
// partial products at part + part_off[l] + s part_stride[l], laid out
// [nout][kin] (the output layer's rows padded to 16); its bias gradient from
// the same products' row sums of dL/dz, bpart + bias_off[l] + s bias_ld[l].
constexpr int kMaxLayers = 17;
struct LayerTab {
    int n;
    long long off_w[kMaxLayers], off_b[kMaxLayers];
    int kin[kMaxLayers], nout[kMaxLayers];
    long long part_off[kMaxLayers], part_stride[kMaxLayers];
    long long bias_off[kMaxLayers];
    int bias_ld[kMaxLayers];
    bf16* wt[kMaxLayers];  // W^T [kin][H] of the hidden layers
};

// BF16 copies of the weights that the products read: W_l^T of every hidden
// layer, the output layer padded to 16 rows and its transpose padded to 64
// columns (the padding is zero from allocation and never written).
__global__ void k_weight_copies(LayerTab t, const float* __restrict__ p, int H, bf16* __restrict__ wout16,
                                bf16* __restrict__ woutT) {
    const int l = blockIdx.y;
    const int kin = t.kin[l];
    const long long n = (long long)t.nout[l] * kin;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(q / kin), i = (int)(q % kin);
        const bf16 v = __float2bfloat16(p[t.off_w[l] + q]);
        if (l < t.n - 1) {
            t.wt[l][(long long)i * H + o] = v;
        } else {
            wout16[(long long)o * H + i] = v;
            woutT[(long long)i * 64 + o] = v;
        }
    }
}

// Weight and bias gradients from the k-split partial products, summed in a
// fixed order (deterministic).
// Weight gradient (o, i) of layer l from its k-split partials.
__device__ __forceinline__ float layer_grad(const LayerTab& t, int l, const float* __restrict__ part, int splits, int o,
                                            int i) {
    float sum = 0.f;
    const float* P = part + t.part_off[l] + (long long)o * t.kin[l] + i;
    for (int s = 0; s < splits; ++s) sum += P[s * t.part_stride[l]];
    return sum;
}

// Bias gradient o of layer l from its partial rows, by one warp: lane k adds
// rows k, k + 32, ..., then a fixed butterfly (the same sum on every lane).
__device__ __forceinline__ float bias_grad_warp(const LayerTab& t, int l, const float* __restrict__ bpart, int brows,
                                                int o, int lane) {
    const float* B = bpart + t.bias_off[l] + o;
    float sum = 0.f;
    for (int r = lane; r < brows; r += 32) sum += B[(long long)r * t.bias_ld[l]];
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    return sum;
}

__global__ void k_reduce_grads(LayerTab t, const float* __restrict__ part, int splits, const float* __restrict__ bpart,
                               int brows, float* __restrict__ g) {
    const int l = blockIdx.y;
    const int kin = t.kin[l], nout = t.nout[l];
    const long long n = (long long)nout * kin;
    const long long q0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
    for (long long q = q0; q < n; q += step) {
        const int o = (int)(q / kin), i = (int)(q % kin);
        g[t.off_w[l] + q] = layer_grad(t, l, part, splits, o, i);
    }
    // biases: one warp each
    const int lane = threadIdx.x & 31;
    for (long long w = q0 >> 5; w < nout; w += step >> 5) {
        const float b = bias_grad_warp(t, l, bpart, brows, (int)w, lane);
        if (lane == 0) g[t.off_b[l] + w] = b;
    }
}

struct AdamArgs {
    float lr, b1, b2, eps, c1, c2;
};

__device__ __forceinline__ float adam_step(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                           long long i, float gi, const AdamArgs& a) {
    const float mi = a.b1 * m[i] + (1.f - a.b1) * gi;
    const float vi = a.b2 * v[i] + (1.f - a.b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - a.lr * (mi / a.c1) / (sqrtf(vi / a.c2) + a.eps);
    p[i] = pi;
    return pi;
}

// One optimiser step of training: the weight and bias gradients summed from
// the k-split partials (fixed order), Adam on them and on the embedding
// (whose gradient is in g), and every BF16 copy the products read (W, W^T,
// the padded output layer).  blockIdx.y: layer, or t.n for the embedding.
__global__ void k_reduce_adam(LayerTab t, const float* __restrict__ part, int splits, const float* __restrict__ bpart,
                              int brows, const float* __restrict__ g, long long off_emb, long long n_emb,
                              float* __restrict__ p, float* __restrict__ am, float* __restrict__ av,
                              bf16* __restrict__ pb, int H, bf16* __restrict__ wout16, bf16* __restrict__ woutT,
                              AdamArgs a) {
    const int l = blockIdx.y;
    const long long step = (long long)gridDim.x * blockDim.x;
    const long long q0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l == t.n) {
        for (long long q = q0; q < n_emb; q += step) {
            const long long i = off_emb + q;
            pb[i] = __float2bfloat16(adam_step(p, am, av, i, g[i], a));
        }
        return;
    }
    const bool out = l == t.n - 1;
    const int kin = t.kin[l], nout = t.nout[l];
    const long long n = (long long)nout * kin;
    const int lane = threadIdx.x & 31;
    for (long long w = q0 >> 5; w < nout; w += step >> 5) {  // biases: one warp each
        const float gb = bias_grad_warp(t, l, bpart, brows, (int)w, lane);
        if (lane == 0) {
            const long long ib = t.off_b[l] + w;
            pb[ib] = __float2bfloat16(adam_step(p, am, av, ib, gb, a));
        }
    }
    for (long long q = q0; q < n; q += step) {
        const int o = (int)(q / kin), i = (int)(q % kin);
        const float sum = layer_grad(t, l, part, splits, o, i);
        const long long iw = t.off_w[l] + (long long)o * kin + i;
        const bf16 w = __float2bfloat16(adam_step(p, am, av, iw, sum, a));
        pb[iw] = w;
        if (!out) {
            t.wt[l][(long long)i * H + o] = w;
        } else {
            wout16[(long long)o * H + i] = w;
            woutT[(long long)i * 64 + o] = w;
        }
    }
}

// ----------------------------------------------------- training samples
// Draw M training samples (antenna, az, za, nu): beams stratified over the
// batch, (az, za, nu) uniform (nu inside the grid's cubic margin), and their
// targets from the gridded beams (Keys cubic in az, za and frequency), as
// sample_item defines them.  A grid-stride loop of 1024-thread blocks (one
// per SM), so that training can run it beside its own launches on the SMs
// those leave free.
constexpr int kSampleThreads = 1024;
__global__ void __launch_bounds__(kSampleThreads, 1)
k_sample(Model m, const float2* __restrict__ grid, SampleRange rg, unsigned long long seed, unsigned long long step,
         int M, int n_out, int* __restrict__ ant, float* __restrict__ az, float* __restrict__ za,
         float* __restrict__ nu, float* __restrict__ T) {
    // every lane of a warp takes the same number of turns (the shuffles need all 32)
    const long long total = (4ll * M * m.n_feed * m.n_ax + 31) / 32 * 32;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride)
        sample_item(m, grid, rg, seed, step, M, n_out, q, ant, az, za, nu, T);
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
    int n_sms = 148;
    int* err = nullptr;   // device status word of the tensor-core products
    // BF16 weight copies for the products (see k_weight_copies)
    std::vector<bf16*> wt;
    bf16* wout16 = nullptr;
    bf16* woutT = nullptr;
    // k-split partial weight gradients (kMaxSplits per layer) and partial bias
    // gradients (four rows per SM per layer)
    float* part = nullptr;
    float* bpart = nullptr;
    LayerTab tab{};
    // work buffers for up to `cap` rows (a multiple of 128)
    long long cap = 0;
    int *ant = nullptr;
    float *az = nullptr, *za = nullptr, *nu = nullptr, *T = nullptr, *Y = nullptr;
    // a second set of training samples: the sampler of step i + 1 runs on a
    // side stream, on SMs the training launches leave free, while step i
    // trains on the other set
    int* ant2 = nullptr;
    float *az2 = nullptr, *za2 = nullptr, *nu2 = nullptr, *T2 = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_time[2] = {nullptr, nullptr};  // timing of the SM splits (surrogate_train)
    std::map<int, int> split_of_batch;             // the split timed fastest, per batch size
    // the fused forward pass's first-layer products (mlp_tc.cu): per live
    // source of one instance (capacity first_cap floats) and per beam
    float* first_P = nullptr;
    float* first_C = nullptr;
    long long first_cap = 0;
    bf16* X0 = nullptr;                      // [cap][d0p]
    std::vector<bf16*> Hs;                   // [cap][H]
    bf16* dY = nullptr;                      // [cap][64] (columns past 16 zero)
    std::vector<bf16*> dZs;                  // [cap][H]: dL/dz of every hidden layer
    double* loss = nullptr;
};

namespace {

constexpr int kMaxSplits = 64;

void sfree(void* p) {
    if (p) cudaFree(p);
}

void free_rows(Surrogate* S) {
    for (void* q : {(void*)S->ant, (void*)S->az, (void*)S->za, (void*)S->nu, (void*)S->T, (void*)S->Y, (void*)S->X0,
                    (void*)S->dY, (void*)S->ant2, (void*)S->az2, (void*)S->za2, (void*)S->nu2, (void*)S->T2})
        sfree(q);
    for (auto* h : S->Hs) sfree(h);
    for (auto* h : S->dZs) sfree(h);
    S->ant = S->ant2 = nullptr;
    S->az = S->za = S->nu = S->T = S->Y = S->az2 = S->za2 = S->nu2 = S->T2 = nullptr;
    S->X0 = S->dY = nullptr;
    S->Hs.assign(S->d.depth, nullptr);
    S->dZs.assign(S->d.depth, nullptr);
    S->cap = 0;
}

// Work buffers for `rows` rows (every array zeroed).
cudaError_t ensure_rows(Surrogate* S, long long rows) {
    if (rows <= S->cap) return cudaSuccess;
    free_rows(S);
    const long long cap = std::max(128ll, (rows + 127) / 128 * 128);
    cudaError_t e = cudaSuccess;
    auto A = [&](void** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(q, bytes);
        if (e == cudaSuccess) e = cudaMemset(*q, 0, bytes);
    };
    const Dims& d = S->d;
    A((void**)&S->ant, sizeof(int) * cap);
    A((void**)&S->az, sizeof(float) * cap);
    A((void**)&S->za, sizeof(float) * cap);
    A((void**)&S->nu, sizeof(float) * cap);
    A((void**)&S->T, sizeof(float) * cap * 8);
    A((void**)&S->Y, sizeof(float) * cap * 8);
    A((void**)&S->ant2, sizeof(int) * cap);
    A((void**)&S->az2, sizeof(float) * cap);
    A((void**)&S->za2, sizeof(float) * cap);
    A((void**)&S->nu2, sizeof(float) * cap);
    A((void**)&S->T2, sizeof(float) * cap * 8);
    A((void**)&S->X0, sizeof(bf16) * cap * d.d0p);
    A((void**)&S->dY, sizeof(bf16) * cap * 64);
    for (int l = 0; l < d.depth; ++l) A((void**)&S->Hs[l], sizeof(bf16) * cap * d.H);
    for (int l = 0; l < d.depth; ++l) A((void**)&S->dZs[l], sizeof(bf16) * cap * d.H);
    if (e == cudaSuccess) S->cap = cap;
    else free_rows(S);
    return e;
}

GemmOperand opnd(const bf16* p, long long ld, long long rows, long long kext, int mn = 0) {
    GemmOperand o;
    o.p = p;
    o.ld = ld;
    o.rows = (int)rows;
    o.kext = (int)kext;
    o.mn = mn;
    return o;
}

// Forward pass of `rows` rows whose features are in X0: hidden layers into
// Hs[l]; then, when training, dL/dy (dY) and the loss, else the FP32 outputs
// Y [rows][8].
cudaError_t forward(Surrogate* S, int rows, bool train, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    cudaError_t e = cudaSuccess;
    const bf16* in = S->X0;
    int kin = d.d0p;
    for (int l = 0; l < d.depth && e == cudaSuccess; ++l) {
        GemmEpi ep{};
        ep.kind = GEPI_RELU;
        ep.out = S->Hs[l];
        ep.ldo = d.H;
        ep.bias = S->p + S->off_b[l];
        e = launch_gemm_tc(opnd(in, kin, S->cap, kin), opnd(S->pb + S->off_w[l], kin, d.H, kin), rows, d.H, 1, false,
                           ep, S->n_sms, S->err, st, L);
        in = S->Hs[l];
        kin = d.H;
    }
    if (e != cudaSuccess) return e;
    GemmEpi ep{};
    ep.bias = S->p + S->off_b[d.depth];
    ep.n_out = d.n_out;
    if (train) {
        ep.kind = GEPI_LOSS;
        ep.out = S->dY;
        ep.ldo = 64;
        ep.target = S->T;
        ep.gscale = 2.f / (float)((long long)rows * d.n_out);
        ep.loss = S->loss;
    } else {
        ep.kind = GEPI_Y;
        ep.out = S->Y;
        ep.ldo = 8;
    }
    return launch_gemm_tc(opnd(in, d.H, S->cap, d.H), opnd(S->wout16, d.H, 16, d.H), rows, 16, 1, false, ep,
                          S->n_sms, S->err, st, L);
}

// k-splits of the weight-gradient products over `rows` rows on `sms` SMs:
// one unit (128-row tile of a product, k-split) per SM, at most kMaxSplits.
int grad_splits(const Surrogate* S, int rows, int sms) {
    const int tiles = 1 + S->d.depth * ((S->d.H + 127) / 128);
    const int kb = (std::max(rows, 64) + 63) / 64;
    return std::max(1, std::min({kMaxSplits, kb, sms / tiles}));
}

// Input gradients for the batch left by forward(train = true), product by
// product: dz_{D-1} = (dY W_out) * (h_{D-1} > 0), dz_{l-1} = (dz_l W_l) *
// (h_{l-1} > 0) into dZs, and the embedding gradient (added into S->g).
cudaError_t input_grads(Surrogate* S, int rows, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    const int D = d.depth, H = d.H;
    const long long cap = S->cap;
    cudaError_t e = cudaSuccess;
    {
        GemmEpi ep{};
        ep.kind = GEPI_MASK;
        ep.out = S->dZs[D - 1];
        ep.ldo = H;
        ep.mask = S->Hs[D - 1];
        ep.ldm = H;
        e = launch_gemm_tc(opnd(S->dY, 64, cap, 64), opnd(S->woutT, 64, H, 64), rows, H, 1, false, ep, S->n_sms,
                           S->err, st, L);
    }
    for (int l = D - 1; l >= 1 && e == cudaSuccess; --l) {
        GemmEpi ep{};
        ep.kind = GEPI_MASK;
        ep.out = S->dZs[l - 1];
        ep.ldo = H;
        ep.mask = S->Hs[l - 1];
        ep.ldm = H;
        e = launch_gemm_tc(opnd(S->dZs[l], H, cap, H), opnd(S->wt[l], H, H, H), rows, H, 1, false, ep, S->n_sms,
                           S->err, st, L);
    }
    if (e == cudaSuccess) {
        // features: only the embedding columns [2F, 2F + E) need a gradient,
        // added into the embedding of each row's beam
        GemmEpi ep{};
        ep.kind = GEPI_EMB;
        ep.ant = S->ant;
        ep.gemb = S->g + S->off_emb;
        ep.emb = d.E;
        const int erows = (d.E + 15) / 16 * 16;
        e = launch_gemm_tc(opnd(S->dZs[0], H, cap, H), opnd(S->wt[0] + (long long)2 * d.F * H, H, erows, H), rows, d.E,
                           1, false, ep, S->n_sms, S->err, st, L);
    }
    return e;
}

// Weight and bias gradients of the batch as k-split partials, from dY, dZs
// and the layer inputs (X0, Hs), all read batch-major: dW_out = dY^T h_{D-1},
// dW_l = dz_l^T x_l, the bias gradients as the row sums of dY^T and dz_l^T;
// with `reduce` the partials are summed into S->g (training sums them in its
// optimiser step instead, k_reduce_adam).
cudaError_t weight_grads(Surrogate* S, int rows, bool reduce, int sms, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    const int D = d.depth, H = d.H;
    // K extent of the products (the batch; TMA reads rows past it as zeros), at
    // least one 64-row box
    const long long kext = std::max(rows, 64);
    const int splits = grad_splits(S, rows, sms);
    cudaError_t e = cudaSuccess;
    if (D + 1 <= kWgradMaxProducts && H <= 256) {
        // every product in one launch
        WgradProduct w[kWgradMaxProducts];
        w[0] = WgradProduct{S->dY, 64, 64, S->Hs[D - 1], H, H, 16, H, S->part + S->tab.part_off[D], H,
                            S->tab.part_stride[D], S->bpart + S->tab.bias_off[D], 16};
        for (int l = 0; l < D; ++l) {
            const int kin = l == 0 ? d.d0p : H;
            w[1 + l] = WgradProduct{S->dZs[l], H, H, l == 0 ? S->X0 : S->Hs[l - 1], kin, kin, H, kin,
                                    S->part + S->tab.part_off[l], kin, S->tab.part_stride[l],
                                    S->bpart + S->tab.bias_off[l], H};
        }
        e = launch_wgrad_tc(w, D + 1, kext, splits, sms, S->err, st, L);
    } else {
        GemmEpi ep{};
        ep.kind = GEPI_F32;
        ep.out = S->part + S->tab.part_off[D];
        ep.ldo = H;
        ep.part_stride = S->tab.part_stride[D];
        ep.bias_part = S->bpart + S->tab.bias_off[D];
        ep.ldo_bias = 16;
        e = launch_gemm_tc(opnd(S->dY, 64, 64, kext, 1), opnd(S->Hs[D - 1], H, H, kext, 1), 16, H, splits, false, ep,
                           sms, S->err, st, L);
        for (int l = D - 1; l >= 0 && e == cudaSuccess; --l) {
            const int kin = l == 0 ? d.d0p : H;
            const bf16* x = l == 0 ? S->X0 : S->Hs[l - 1];
            GemmEpi epl{};
            epl.kind = GEPI_F32;
            epl.out = S->part + S->tab.part_off[l];
            epl.ldo = kin;
            epl.part_stride = S->tab.part_stride[l];
            epl.bias_part = S->bpart + S->tab.bias_off[l];
            epl.ldo_bias = H;
            e = launch_gemm_tc(opnd(S->dZs[l], H, H, kext, 1), opnd(x, kin, kin, kext, 1), H, kin, splits, false, epl,
                               sms, S->err, st, L);
        }
    }
    if (e == cudaSuccess && reduce) {
        k_reduce_grads<<<dim3(64, D + 1), 256, 0, st>>>(S->tab, S->part, splits, S->bpart, splits, S->g);
        ++*L;
        e = cudaGetLastError();
    }
    return e;
}

// One training pass over the `rows` samples in S->ant / az / za / nu / T; the
// loss is accumulated into S->loss, which the caller zeroes.  Leaves the
// gradients of the loss as k-split partials and the embedding gradient in
// S->g, with `reduce` every gradient summed into S->g.  Where the network's
// shape allows, the row-local part (features, forward, loss, input gradients,
// embedding gradient) is one fused launch (mlp_chain_tc.cu); else it runs
// kernel by kernel.  The weight gradients follow as products over the batch.
// The tensor-core launches take at most `sms` SMs.
cudaError_t train_rows(Surrogate* S, int rows, bool reduce, int sms, cudaStream_t st, long long* L) {
    const Dims& d = S->d;
    const int D = d.depth, H = d.H;
    // the embedding gradient accumulates; the rest is written by the reduction
    cudaError_t e = reduce ? cudaMemsetAsync(S->g, 0, sizeof(float) * (size_t)S->n_par, st)
                           : cudaMemsetAsync(S->g + S->off_emb, 0, sizeof(float) * (size_t)(S->n_par - S->off_emb), st);
    const long long kext = std::max(rows, 64);
    if (e == cudaSuccess && kext > rows) {
        // a batch below 64 rows: the rows [rows, 64) the box reads must be zero in every operand
        auto zero = [&](bf16* a, int width) {
            if (e == cudaSuccess)
                e = cudaMemsetAsync(a + (long long)rows * width, 0, sizeof(bf16) * (size_t)(kext - rows) * width, st);
        };
        zero(S->X0, d.d0p);
        for (int l = 0; l < D; ++l) zero(S->Hs[l], H);
        zero(S->dY, 64);
        for (int l = 0; l < D; ++l) zero(S->dZs[l], H);
    }
    if (e != cudaSuccess) return e;
    if (mlp_chain_supported(d.F, d.E, H, D, d.d0p, d.n_out, rows)) {
        ChainArgs c{};
        c.F = d.F; c.E = d.E; c.H = H; c.depth = D; c.d0p = d.d0p; c.n_out = d.n_out;
        c.nu_mid = d.nu_mid; c.nu_half = d.nu_half;
        c.M = rows;
        c.p = S->p;
        for (int l = 0; l <= D; ++l) c.off_b[l] = S->off_b[l];
        c.off_emb = S->off_emb;
        c.Bf = S->Bf;
        for (int l = 0; l < D; ++l) {
            c.w[l] = S->pb + S->off_w[l];
            c.wt[l] = S->wt[l];
            c.Hs[l] = S->Hs[l];
            c.dZs[l] = S->dZs[l];
        }
        c.wout16 = S->wout16;
        c.woutT = S->woutT;
        c.ant = S->ant; c.az = S->az; c.za = S->za; c.nu = S->nu; c.T = S->T;
        c.X0 = S->X0;
        c.dY = S->dY;
        c.gscale = 2.f / (float)((long long)rows * d.n_out);
        c.loss = S->loss;
        c.gemb = S->g + S->off_emb;
        e = launch_mlp_chain_tc(c, sms, S->err, st, L);
    } else {
        e = launch_features(d, S->Bf, S->p + S->off_emb, rows, S->ant, S->az, S->za, S->nu, S->X0, nullptr, 0, st);
        ++*L;
        if (e == cudaSuccess) e = forward(S, rows, true, st, L);
        if (e == cudaSuccess) e = input_grads(S, rows, st, L);
    }
    if (e == cudaSuccess) e = weight_grads(S, rows, reduce, sms, st, L);
    return e;
}

cudaError_t weight_copies(Surrogate* S, cudaStream_t st, long long* L) {
    k_weight_copies<<<dim3(64, S->d.depth + 1), 256, 0, st>>>(S->tab, S->p, S->d.H, S->wout16, S->woutT);
    if (L) ++*L;
    return cudaGetLastError();
}

cudaError_t check_err(Surrogate* S, cudaStream_t st) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, S->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h != 0) {
        cudaMemsetAsync(S->err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return cudaErrorLaunchTimeout;
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
    d.d0p = std::max(64, (d.d0 + 31) / 32 * 32);  // one 64-column panel at least
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
    if (e == cudaSuccess) e = cudaMalloc(&S->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(S->err, 0, sizeof(int));
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->n_sms, cudaDevAttrMultiProcessorCount, dev);
    // BF16 weight copies and the layer table of the products
    S->wt.assign(depth, nullptr);
    LayerTab& t = S->tab;
    t.n = depth + 1;
    long long part = 0;
    for (int l = 0; l <= depth; ++l) {
        const bool out = l == depth;
        const int kin = l == 0 ? d.d0p : H;
        t.off_w[l] = S->off_w[l];
        t.off_b[l] = S->off_b[l];
        t.kin[l] = kin;
        t.nout[l] = out ? 8 : H;
        t.part_off[l] = part;
        t.part_stride[l] = out ? (long long)H * 16 : (long long)H * kin;
        part += kMaxSplits * t.part_stride[l];
        t.bias_ld[l] = out ? 16 : H;
        t.bias_off[l] = (long long)l * kMaxSplits * H;
        if (!out && e == cudaSuccess) {
            e = cudaMalloc(&S->wt[l], sizeof(bf16) * (size_t)kin * H);
            t.wt[l] = S->wt[l];
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&S->part, sizeof(float) * (size_t)part);
    if (e == cudaSuccess) e = cudaMalloc(&S->bpart, sizeof(float) * (size_t)(depth + 1) * kMaxSplits * H);
    if (e == cudaSuccess) e = cudaMalloc(&S->wout16, sizeof(bf16) * 16 * (size_t)H);
    if (e == cudaSuccess) e = cudaMemset(S->wout16, 0, sizeof(bf16) * 16 * (size_t)H);
    if (e == cudaSuccess) e = cudaMalloc(&S->woutT, sizeof(bf16) * 64 * (size_t)H);
    if (e == cudaSuccess) e = cudaMemset(S->woutT, 0, sizeof(bf16) * 64 * (size_t)H);
    if (e == cudaSuccess) {
        k_to_bf16<<<gridsz(o, 256), 256>>>(o, S->p, S->pb);
        e = weight_copies(S, 0, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
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
    free_rows(S);
    if (S->side) cudaStreamDestroy(S->side);
    for (int i = 0; i < 2; ++i) {
        if (S->ev_ready[i]) cudaEventDestroy(S->ev_ready[i]);
        if (S->ev_free[i]) cudaEventDestroy(S->ev_free[i]);
        if (S->ev_time[i]) cudaEventDestroy(S->ev_time[i]);
    }
    for (void* q : {(void*)S->p, (void*)S->g, (void*)S->am, (void*)S->av, (void*)S->pb, (void*)S->Bf, (void*)S->loss,
                    (void*)S->err, (void*)S->part, (void*)S->bpart, (void*)S->wout16, (void*)S->woutT,
                    (void*)S->first_P, (void*)S->first_C})
        sfree(q);
    for (auto* w : S->wt) sfree(w);
    delete S;
}

long long surrogate_param_count(const Surrogate* S) { return S->n_par; }
long long surrogate_eval_bytes(const Surrogate* S) {
    return S->n_par * (long long)(sizeof(float) + sizeof(bf16)) + (long long)S->hB.size() * (long long)sizeof(float);
}
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
        e = weight_copies(S, 0, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
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
    e = train_rows(S, n, true, S->n_sms, st, &L);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grads_host, S->g, sizeof(float) * S->n_par, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, S->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = check_err(S, st);
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
    e = launch_features(d, S->Bf, S->p + S->off_emb, n, S->ant, S->az, S->za, S->nu, S->X0, nullptr, 0, st);
    if (e == cudaSuccess) e = forward(S, n, false, st, &L);
    if (e != cudaSuccess) return e;
    std::vector<float> y((size_t)n * 8);
    e = cudaMemcpyAsync(y.data(), S->Y, sizeof(float) * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = check_err(S, st);
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
    // frequencies inside the grid's cubic margin: fractional index in [1, n_nu - 3)
    const SampleRange rg{1.f, (float)(m.n_nu - 4) * 0.999999f, (float)nu0, (float)dnu};
    if (!S->side) {
        e = cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&S->ev_ready[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_free[i], cudaEventDisableTiming);
        }
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&S->ev_time[i]);
        if (e != cudaSuccess) return e;
    }
    // SMs: the training launches take at most `sms` (one CTA per SM each), the
    // sampler of the next step one block on each of the others (a 1024-thread
    // block does not fit beside a training CTA, so neither waits for the
    // other).  Candidate splits: the fewest SMs that walk the batch's 128-row
    // tiles in the fewest rounds (leaving at least 8 to the sampler), every SM
    // but 8, the fewest for one round more (more SMs for the sampler), and the
    // fewest for the rounds two thirds of the SMs take when that is over 4
    // (the sampler's time grows with the batch over its SMs, so large batches
    // balance near there).
    // With enough steps each runs three steps, the last two timed (their
    // samples drawn beside the same split), and the fastest stays (and is
    // kept for later calls with this batch size).
    const int tiles = (batch + 127) / 128;
    const int most = std::max(1, S->n_sms - 8);
    auto split_for = [&](int rounds) { return std::min(most, std::max(1, (tiles + rounds - 1) / rounds)); };
    const int r0 = (tiles + most - 1) / most;
    const int two_thirds = std::max(1, 2 * S->n_sms / 3);
    const int r23 = (tiles + two_thirds - 1) / two_thirds;
    int cand[4], nc = 0;
    for (int b : {split_for(r0), most, split_for(r0 + 1), r0 > 4 ? split_for(r23) : split_for(r0)}) {
        bool seen = false;
        for (int i = 0; i < nc; ++i) seen = seen || cand[i] == b;
        if (!seen) cand[nc++] = b;
    }
    const auto known = S->split_of_batch.find(batch);
    const bool tune = known == S->split_of_batch.end() && nc > 1 && steps >= 3 * nc + 3;
    int sms = known != S->split_of_batch.end() ? known->second : cand[0], best = 0;
    float t_best = 0.f;
    // sample sets: set 0 the arrays the training pass reads, set 1 the second
    // one; the pointers swap every step
    int* s_ant[2] = {S->ant, S->ant2};
    float* s_az[2] = {S->az, S->az2};
    float* s_za[2] = {S->za, S->za2};
    float* s_nu[2] = {S->nu, S->nu2};
    float* s_T[2] = {S->T, S->T2};
    auto sample = [&](int it, int blocks) {  // on the side stream, into set it & 1, once the set is free
        const int k = it & 1;
        cudaError_t x = cudaSuccess;
        if (it >= 2) x = cudaStreamWaitEvent(S->side, S->ev_free[k], 0);
        if (x == cudaSuccess) {
            k_sample<<<blocks, kSampleThreads, 0, S->side>>>(m, grid, rg, seed, (unsigned long long)it, batch,
                                                             d.n_out, s_ant[k], s_az[k], s_za[k], s_nu[k], s_T[k]);
            ++*L;
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) x = cudaEventRecord(S->ev_ready[k], S->side);
        return x;
    };
    // the side stream starts after the work already queued on st; the first
    // samples take every SM
    e = cudaEventRecord(S->ev_free[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->side, S->ev_free[0], 0);
    if (e == cudaSuccess) e = sample(0, S->n_sms);
    for (int it = 0; it < steps && e == cudaSuccess; ++it) {
        const int k = it & 1;
        if (tune && it > 0 && it <= 3 * nc && it % 3 == 0) {
            // steps it - 2 and it - 1 ran candidate it / 3 - 1, timed
            const int c = it / 3 - 1;
            float ms = 0.f;
            e = cudaEventSynchronize(S->ev_time[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, S->ev_time[0], S->ev_time[1]);
            if (c == 0 || ms < t_best) {
                t_best = ms;
                best = c;
            }
            sms = it < 3 * nc ? cand[it / 3] : cand[best];
            if (it == 3 * nc) S->split_of_batch[batch] = sms;
        }
        if (e == cudaSuccess && tune && it < 3 * nc && it % 3 == 1) e = cudaEventRecord(S->ev_time[0], st);
        if (e != cudaSuccess) break;
        // the next step's sampler runs beside this step's training launches
        if (it + 1 < steps && (e = sample(it + 1, S->n_sms - sms)) != cudaSuccess) break;
        S->ant = s_ant[k];
        S->az = s_az[k];
        S->za = s_za[k];
        S->nu = s_nu[k];
        S->T = s_T[k];
        if (it == 0 || it == steps - 1) e = cudaMemsetAsync(S->loss, 0, sizeof(double), st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, S->ev_ready[k], 0);
        if (e == cudaSuccess) e = train_rows(S, batch, false, sms, st, L);
        if (e == cudaSuccess) e = cudaEventRecord(S->ev_free[k], st);  // set k read for the last time
        if (e != cudaSuccess) break;
        if (it == 0 || it == steps - 1) {
            double l = 0;
            e = cudaMemcpyAsync(&l, S->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            l /= (double)batch * d.n_out;
            if (it == 0) *loss_first = l;
            if (it == steps - 1) *loss_last = l;
        }
        if (e != cudaSuccess) break;
        AdamArgs a;
        a.lr = lr1 + 0.5f * (lr0 - lr1) * (1.f + cosf((float)kPi * it / std::max(1, steps - 1)));
        S->adam_k += 1;
        a.b1 = 0.9f;
        a.b2 = 0.999f;
        a.eps = 1e-8f;
        a.c1 = 1.f - powf(0.9f, (float)S->adam_k);
        a.c2 = 1.f - powf(0.999f, (float)S->adam_k);
        const long long n_emb = S->n_par - S->off_emb;
        const long long max_layer = (long long)std::max(d.d0p, d.H) * (d.H + 1);
        const int splits = grad_splits(S, batch, sms);
        k_reduce_adam<<<dim3(gridsz(std::max(max_layer, n_emb), 256), d.depth + 2), 256, 0, st>>>(
            S->tab, S->part, splits, S->bpart, splits, S->g, S->off_emb, n_emb, S->p, S->am, S->av, S->pb, d.H,
            S->wout16, S->woutT, a);
        ++*L;
        e = cudaGetLastError();
        if (e == cudaSuccess && tune && it < 3 * nc && it % 3 == 2) e = cudaEventRecord(S->ev_time[1], st);
    }
    // the arrays back in their places (set 0 first), whatever step ended last
    S->ant = s_ant[0];
    S->az = s_az[0];
    S->za = s_za[0];
    S->nu = s_nu[0];
    S->T = s_T[0];
    S->ant2 = s_ant[1];
    S->az2 = s_az[1];
    S->za2 = s_za[1];
    S->nu2 = s_nu[1];
    S->T2 = s_T[1];
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->side);
    if (e == cudaSuccess) e = check_err(S, st);
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
    // the fused tensor-core forward pass (the first layer's source and beam
    // parts computed once each, then the layers and WA in one launch per
    // instance) where the network shape allows, else the network's
    // layer-by-layer tensor-core products
    const bool tc = mlp_tc_supported(d.F, d.E, d.H, d.depth, d.d0p, d.n_out);
    MlpTcArgs ta{};
    cudaError_t e = cudaSuccess;
    if (tc) {
        ta.F = d.F; ta.E = d.E; ta.H = d.H; ta.depth = d.depth; ta.d0p = d.d0p; ta.n_beam = d.n_ant;
        ta.n_out = d.n_out; ta.nu_mid = d.nu_mid; ta.nu_half = d.nu_half;
        ta.p = S->p; ta.pb = S->pb; ta.off_emb = S->off_emb; ta.Bf = S->Bf;
        for (int l = 0; l <= d.depth; ++l) { ta.off_w[l] = S->off_w[l]; ta.off_b[l] = S->off_b[l]; }
        // the first-layer products: P per live source (grown to the largest
        // live count of the call), C per beam from the current parameters
        long long max_live = 0;
        for (int j = 0; j < n_inst; ++j) max_live = std::max(max_live, (long long)h_nlive[h_inst[inst0 + j].t]);
        const long long need = mlp_tc_first_floats(d.H, max_live);
        if (need > S->first_cap) {
            sfree(S->first_P);
            S->first_P = nullptr;
            S->first_cap = 0;
            e = cudaMalloc((void**)&S->first_P, sizeof(float) * (size_t)need);
            if (e == cudaSuccess) S->first_cap = need;
        }
        if (e == cudaSuccess && !S->first_C) e = cudaMalloc((void**)&S->first_C, sizeof(float) * (size_t)d.n_ant * d.H);
        ta.P = S->first_P;
        ta.C = S->first_C;
        if (e == cudaSuccess) e = launch_mlp_beam_first(ta, st, L);
    } else {
        e = ensure_rows(S, chunk);
    }
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
            e = launch_features(d, S->Bf, S->p + S->off_emb, R, S->ant, S->az, S->za, S->nu, S->X0, nullptr, 0, st);
            *L += 2;
            if (e == cudaSuccess) e = forward(S, R, false, st, L);
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
