// common.cuh -- shared declarations of the matvis GB300 library (device and
// host side).  Nothing here is part of the public C-ABI (include/matvis.h).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

namespace mv {

constexpr double kCLight = 299792458.0;   // m/s
constexpr double kPi = 3.14159265358979323846;

// Column padding of the Z matrix along the source axis: every instance's
// K = n_ax * n_live is rounded up to a multiple of this (the tensor-core
// HERK's TMEM flush granularity is a multiple of its 64-wide k-blocks).
constexpr int kKPad = 256;

// Device-side error codes written into the context's status word.
enum DevErr : int { kDevOk = 0, kDevTimeout = 1, kDevBadArg = 2 };

// ----------------------------------------------------------------- tables
// One (time, frequency) instance of a simulate call.
struct Inst {
    int t;            // index into the call's distinct times (live tables)
    int c;            // index into the call's distinct channels
    long long v_off;  // offset of this instance's V in complex64 elements
};

// One channel of a simulate call.
struct Chan {
    double kappa;     // nu / c  (turns of phase per metre of path difference)
    float ln_ratio;   // ln(nu / nu_ref)
    int m0;           // first frequency node of the beam-grid stencil
    float w[4];       // frequency stencil weights (Keys cubic)
};

// Live-source tables of the distinct times of a call (structure of arrays,
// one row of pitch `pitch` per time).
struct LiveTables {
    double* e;        // [n_times][pitch] East component of s_hat
    double* n;        // North
    double* u;        // Up
    // s_hat in fixed point for the phase (NULL: not written): component c of
    // live source s at time t is sfix[(3 t + c) pitch + s] = S + 2^31 with
    // S = rint(s_c 2^31) (clamped to int32), and seps[...] = s_c - S 2^-31
    unsigned* sfix;
    float* seps;
    int* idx;         // catalogue index of each live source
    float2* azza;     // (az, za) radians, FP32
    int* n_live;      // [n_times]
    long long pitch;
};

// Static description of the sky / array / beam on the device.
struct Model {
    // sky
    long long n_src;
    const double* xeq;       // [3][n_src] SoA: x, y, z (eq. "xeq")
    const float* sqrt_flux;  // [n_src] sqrt(flux at nu_ref)
    const float* half_alpha; // [n_src] spectral index / 2
    const float4* pol_m;     // [n_src] (m00, Re m10, Im m10, m11) of C = M M^dagger at nu_ref, or NULL
    // array
    int n_ant;
    const double* ant_e;     // [n_ant]
    const double* ant_n;
    const double* ant_u;
    const int* beam_idx;     // [n_ant]
    // beam
    int beam_kind;           // 1 gaussian, 2 grid
    float gauss_c;           // 4 ln2 / fwhm^2
    int n_beam, n_feed, n_ax;
    int n_nu, n_za, n_az;
    float dza, daz;
    int interp;              // 0 cubic, 1 bilinear
};

// A tile of a listed cover (the redundant-baseline expansion): A rows [r0,
// r0 + 128) and B rows [c0, c0 + ncol) of U; its entries with a row >= rlim
// or a column >= clim belong to no block of the cover.
struct TileDesc {
    int r0, c0, ncol, rlim, clim, pad0, pad1, pad2;
};

// What the tensor-core HERK writes: the full V (uidx NULL), or one value per
// redundant group, V_u[inst][g][p][q]: uidx[a * n_ant + b] (antennas in the
// cover's order) = 2 g + conj where entry (a, b) of V computes group g's
// representative (conj: the representative is its conjugate), else -1.  tl:
// the tiles of the cover (NULL: the lower triangle), n_tl of them.
struct HerkOut {
    const TileDesc* tl;
    int n_tl;
    const int* uidx;
    int n_ant, n_feed;
};

// ------------------------------------------------------------ host launchers
// (defined in the .cu files; all enqueue on `st` and return the CUDA error)
cudaError_t launch_cull(const Model& m, const double* d_R, int n_times, LiveTables lt,
                        int* d_counts, int* d_offsets, int blocks_per_time, cudaStream_t st,
                        long long* launches);
cudaError_t launch_beam_planes(const Model& m, const float2* d_grid, const Chan* d_chan, int n_chan,
                               float2* d_planes, cudaStream_t st, long long* launches);
// Z-side source factor of a polarised sky (eq. "fullz"): the two axis
// components a0, a1 of one (beam, feed) times M = [[m00, 0], [m10, m11]] and
// the spectral factor w: z0 = w (a0 m00 + a1 m10), z1 = w a1 m11.
__device__ __forceinline__ void apply_sky_sqrt(float2 a0, float2 a1, float4 M, float w, float2& z0, float2& z1) {
    z0.x = w * (a0.x * M.x + (a1.x * M.y - a1.y * M.z));
    z0.y = w * (a0.y * M.x + (a1.x * M.z + a1.y * M.y));
    z1.x = w * (a1.x * M.w);
    z1.y = w * (a1.y * M.w);
}

// WA[slot] = sqrt(I_s) A(s) for the live sources and zero for the rest of
// the pitch; amax[slot] (zeroed by the caller) receives max |WA| over the
// slot's components, as float bits.
cudaError_t launch_wa(const Model& m, const float2* d_planes, const Chan* d_chan, const Inst* d_inst,
                      int inst0, int n_inst, LiveTables lt, float2* d_wa, long long wa_pitch,
                      float* d_amax, cudaStream_t st, long long* launches);
// A group of instances of one time whose Z matrices are built together (the
// FP64 path length x_a . s_hat is formed once per antenna and source).
struct ZGroup {
    int inst0;        // first instance (into the call's instance table)
    int n;            // instances in the group (same time, consecutive)
    int slot0;        // workspace slot of the first instance
    int uniform;      // channels are equally spaced: kappa_j = kappa0 + j dkappa
    double kappa0, dkappa;
};
// Largest number of instances of one batch (channels of one time, or pairs).
constexpr int kMaxBatch = 256;

// Antenna factor of the fixed-point phase for one wavenumber kappa (turns per
// metre): y_c = kappa x_a,c, Y_c = rint(y_c 2^32) = yh_c 2^32 + yl_c (yl
// unsigned), yf_c = (float) y_c, negk = -sum_c yl_c 2^31 mod 2^64.  With
// the source's S_c + 2^31 and residual eps_c (LiveTables) the phase
// frac(kappa x_a . s_hat) follows from integer multiply-adds (zbuild.cu).
struct alignas(16) AntPhase {
    unsigned yl[3];
    int yh[3];
    float yf[3];
    unsigned negk_lo, negk_hi, pad;
};

// Z build of a batch of groups: writes FP32 planes (prec 0) or scaled FP16
// hi/lo planes (prec 2) of U into workspace slots.
// Everything the Z build of one batch needs, for Z-build warps running
// inside another kernel (the HERK of the previous batch).
struct ZJob {
    Model m;
    const Inst* inst;
    const ZGroup* groups;
    int g_first, n_groups;
    LiveTables lt;
    const float2* wa;
    long long wa_pitch;
    const float* amax;
    void* u;
    void* ulo;
    int rows;
    long long k_pitch;
    const AntPhase* aph;
    int n_phase;
};

// Antenna phase table of a batch (the first half of launch_zbuild); with
// d_amax (FP16 planes) it also gives every instance of a Z group the group's
// max |WA|, so that one FP16 scale serves the whole group.
cudaError_t launch_ant_phase(const Model& m, const Inst* d_inst, const Chan* d_chan, const ZGroup* d_groups,
                             int g_first, int n_groups, AntPhase* d_aph, int n_phase, float* d_amax,
                             cudaStream_t st, long long* launches);

// d_aph: workspace for n_groups x n_phase x n_ant AntPhase entries, n_phase
// >= max(2, largest group of the batch).
cudaError_t launch_zbuild(const Model& m, const Inst* d_inst, const Chan* d_chan, const ZGroup* d_groups,
                          int g_first, int n_groups, LiveTables lt, const float2* d_wa, long long wa_pitch,
                          float* d_amax, void* d_u, void* d_u_lo, int prec, int rows,
                          long long k_pitch, int max_blocks, AntPhase* d_aph, int n_phase, cudaStream_t st,
                          long long* launches);
cudaError_t launch_herk_fp32(const Inst* d_inst, int inst0, int n_inst, LiveTables lt, int n_ax,
                             const float* d_u, int rows, long long k_pitch, float2* d_v, int N,
                             int flush_k, cudaStream_t st, long long* launches);
// Persistent tensor-core HERK over n_inst instance slots: tiles 128 x bn
// (bn = 128 or 256), the source axis split `split` ways (split > 1 writes
// 128 x bn FP32 partial tiles, summed by a finalize kernel), TMEM flushed into
// FP32 sums every flush_kblocks k-blocks.  d_sched holds n_inst + 1 ints
// (instance order and the work counter).  zj (optional, see
// herk_tc_fusable): the Z build of the next batch, run by extra warps of the
// same launch on every SM.
cudaError_t launch_herk_tc(const Inst* d_inst, int inst0, int n_inst, LiveTables lt, int n_ax,
                           const __nv_bfloat16* d_hi, const __nv_bfloat16* d_lo, int rows,
                           long long k_pitch, int n_slots, int fp16, const float* d_amax, float2* d_v,
                           int N, int flush_kblocks, int split, int bn, int n_ctas, int* d_sched,
                           float* d_partial, int* d_err, const ZJob* zj, int zprec, const HerkOut* out,
                           cudaStream_t st, long long* launches);
// One bounded mbarrier wait that nothing completes, with a limit of limit_s
// (<= 10 s): records kDevTimeout in d_err (self-test of the failure path).
cudaError_t launch_wait_probe(int* d_err, double limit_s, cudaStream_t st);
// Whether the HERK can carry the Z build (tile width 128; one feed and one
// axis, or two and two; FP16x3).
bool herk_tc_fusable(int bn, int zprec, int n_ax, int n_feed);
// Set kernel attributes of the tensor-core HERK (once per process, outside
// any stream capture).
cudaError_t herk_tc_init();
// Work units of that HERK (each needs 128 x bn x 4 bytes of partials when split > 1).
int herk_tc_units(int rows, int n_slots, int split, int bn);
bool herk_tc_available();

// Set the message mv_last_error() returns on this thread.
void set_last_error(const char* msg);

// ------------------------------------------------------ learned beam (mlp.cu)
struct Surrogate;
Surrogate* surrogate_create(int F, int E, int H, int depth, int n_out, int n_ant, float s_az, float s_za, float s_nu,
                            unsigned long long seed, double nu_mid, double nu_half, cudaError_t* err);
void surrogate_destroy(Surrogate* S);
long long surrogate_param_count(const Surrogate* S);
// Device bytes the surrogate's evaluation reads: FP32 parameters (biases,
// embedding), their BF16 copy (weights) and the Fourier matrix.
long long surrogate_eval_bytes(const Surrogate* S);
int surrogate_fourier(const Surrogate* S, float* out);
void surrogate_layout(const Surrogate* S, long long* off_w, long long* off_b, long long* off_emb, int* d0p);
cudaError_t surrogate_get_params(const Surrogate* S, float* host);
cudaError_t surrogate_set_params(Surrogate* S, const float* host);
cudaError_t surrogate_grad(Surrogate* S, int n, const int* ant, const float* az, const float* za, const float* nu,
                           const float* T, float* grads_host, double* loss, cudaStream_t st);
cudaError_t surrogate_eval(Surrogate* S, int n, const int* ant, const float* az, const float* za, const float* nu,
                           float* out_host, cudaStream_t st);
cudaError_t surrogate_train(Surrogate* S, const Model& m, const float2* grid, double nu0, double dnu, int steps,
                            int batch, float lr0, float lr1, unsigned long long seed, cudaStream_t st,
                            double* loss_first, double* loss_last, long long* L);
cudaError_t surrogate_wa(Surrogate* S, const Model& m, const std::vector<Inst>& h_inst, int inst0, int n_inst,
                         const std::vector<int>& h_nlive, const std::vector<double>& h_nu, double nu_ref,
                         LiveTables lt, float2* wa, long long wa_pitch, float* amax, int* d_err, int n_sms,
                         cudaStream_t st, long long* L);

// The network of a surrogate, for the tensor-core forward pass (mlp_tc.cu).
struct MlpTcArgs {
    int F, E, H, depth, d0p, n_beam, n_out;
    float nu_mid, nu_half;
    const float* p;               // FP32 parameters (biases, embedding)
    const __nv_bfloat16* pb;      // BF16 copy (weights)
    long long off_w[9], off_b[9];  // per layer: hidden layers, then the output layer
    long long off_emb;
    const float* Bf;              // Fourier matrix [F][3]
    float* P;                     // per live source: W_0's Fourier columns times the features
                                  // (mlp_tc_first_floats(H, live count) floats)
    float* C;                     // per beam: W_0's embedding columns times e_b, plus b_0 ([n_beam][H])
};
// Whether the tensor-core forward pass handles this network shape.
bool mlp_tc_supported(int F, int E, int H, int depth, int d0p, int n_out);
cudaError_t mlp_tc_init();
// Floats of MlpTcArgs::P for instances of up to max_live live sources.
long long mlp_tc_first_floats(int H, long long max_live);
// MlpTcArgs::C from the current parameters (once per set of parameters).
cudaError_t launch_mlp_beam_first(const MlpTcArgs& a, cudaStream_t st, long long* launches);
// WA of one instance (live count K at time index t, frequency nu) from the
// network: rows (beam b, source s), b < n_beam; WA[b][comp][s] as launch_wa.
// Computes the instance's P, then runs the fused pass; C must be current.
cudaError_t launch_mlp_wa_tc(const MlpTcArgs& a, const Model& m, LiveTables lt, int t, int K, float nu,
                             float ln_ratio, float2* wa_slot, long long wa_pitch, float* amax, int* d_err,
                             int n_sms, cudaStream_t st, long long* launches);

// ------------------------------ fused training pass (mlp_chain_tc.cu)
// One training batch of the surrogate through every row-local step in one
// launch: features, the hidden layers, the output layer with the loss and
// dL/dy, the input gradients back through the layers with the ReLU masks,
// and the embedding gradient.  The weight gradients (products over the batch)
// are left to the tensor-core products below, which read what this pass
// stores: X0, every H_l, dY and every dZ_l, batch-major.
constexpr int kChainMaxLayers = 5;  // deeper networks run product by product
struct ChainArgs {
    int F, E, H, depth, d0p, n_out;
    float nu_mid, nu_half;
    int M;                                       // rows of the batch
    const float* p;                              // FP32 parameters (biases, embedding)
    long long off_b[kChainMaxLayers + 1];        // hidden layers, then the output layer
    long long off_emb;
    const float* Bf;                             // Fourier matrix [F][3]
    const __nv_bfloat16* w[kChainMaxLayers];     // W_l [H][kin_l] (BF16)
    const __nv_bfloat16* wout16;                 // W_out [16][H], rows past n_out zero
    const __nv_bfloat16* woutT;                  // W_out^T [H][64], columns past n_out zero
    const __nv_bfloat16* wt[kChainMaxLayers];    // W_l^T [kin_l][H]
    const int* ant;                              // samples: beam, az, za, nu, targets [M][n_out]
    const float *az, *za, *nu, *T;
    __nv_bfloat16* X0;                           // [M][d0p]
    __nv_bfloat16* Hs[kChainMaxLayers];          // [M][H]
    __nv_bfloat16* dY;                           // [M][64]: columns [0, 16) written
    __nv_bfloat16* dZs[kChainMaxLayers];         // [M][H]
    float gscale;                                // dL/dy = gscale (y - target)
    double* loss;                                // sum of squared residuals (atomic)
    float* gemb;                                 // [n_beam][E] embedding gradient (atomic)
};
// Whether the fused pass handles this network shape and batch.
bool mlp_chain_supported(int F, int E, int H, int depth, int d0p, int n_out, int M);
cudaError_t mlp_chain_init();
// n_sms: the SMs the launch may take (one CTA each, as few as keep the same
// number of tiles per CTA).
cudaError_t launch_mlp_chain_tc(const ChainArgs& a, int n_sms, int* d_err, cudaStream_t st, long long* launches);

// ------------------------------- weight gradients in one launch (mlp_wgrad_tc.cu)
// dW = A^T X and db = A^T 1 over a batch of kext rows for several layers at
// once, as FP32 partials per k-split (the batch cut into `splits` ranges).
// A: dL/dz [kext][lda] (a_rows columns, at least M and 64); X: the layer's
// input [kext][ldb] (b_rows columns, at least N and 64, N <= 256); BF16,
// 16-byte aligned rows; rows of either past kext read as zero.  Partial s of
// dW[m][n] at out + s part_stride + m ldo + n, of db[m] at bias_part + s
// ldo_bias + m.
constexpr int kWgradMaxProducts = kChainMaxLayers + 1;
struct WgradProduct {
    const __nv_bfloat16* A;
    long long lda;
    int a_rows;
    const __nv_bfloat16* X;
    long long ldb;
    int b_rows;
    int M, N;
    float* out;
    long long ldo, part_stride;
    float* bias_part;
    long long ldo_bias;
};
cudaError_t wgrad_tc_init();
cudaError_t launch_wgrad_tc(const WgradProduct* p, int n_prod, long long kext, int splits, int n_sms, int* d_err,
                            cudaStream_t st, long long* launches);

// ------------------------------------- tensor-core products (mlp_train_tc.cu)
// A BF16 operand of rows (M or N) x kext (K).  K-major (mn = 0): a
// [rows][ld] array, K contiguous.  MN-major (mn = 1): a [kext][ld] array, the
// rows dimension contiguous (the transpose, read without a transposed copy).
// ld and the base 16-byte aligned; entries past kext (or rows) read as zero.
struct GemmOperand {
    const __nv_bfloat16* p;
    long long ld;
    int rows, kext;
    int mn;
};
// Fused epilogue of D = A B^T (see mlp_train_tc.cu).
enum GemmEpiKind : int { GEPI_RELU = 0, GEPI_LOSS = 1, GEPI_MASK = 2, GEPI_F32 = 3, GEPI_EMB = 4, GEPI_Y = 5 };
struct GemmEpi {
    int kind;
    void* out;                   // rows of D: BF16 (RELU, MASK, LOSS) or FP32 (F32, Y)
    long long ldo;
    __nv_bfloat16* outT;         // columns of D as rows (RELU, MASK: may be NULL; LOSS: 16 rows)
    long long ldt;
    const float* bias;           // RELU, LOSS, Y
    const __nv_bfloat16* mask;   // MASK: h_prev, rows of ldm
    long long ldm;
    const float* target;         // LOSS: [M][n_out]
    int n_out;                   // LOSS, Y
    float gscale;                // LOSS: dL/dy = gscale (y - target)
    double* loss;                // LOSS: sum of squared residuals (atomic)
    const int* ant;              // EMB: beam of each row
    float* gemb;                 // EMB: [n_beam][emb] (atomic)
    int emb;
    long long part_stride;       // F32: elements between the partials of two k-splits
    float* bias_part;            // F32 (may be NULL): row sums of A over each k-split's K range,
    long long ldo_bias;          // [split][M] at bias_part + split ldo_bias
};
cudaError_t gemm_tc_init();
// D[M][N] = A[M][K] B[N][K]^T on tcgen05 with the epilogue e; the K axis is
// cut into `splits` ranges (F32 writes one partial per range); two_row_tiles:
// 256-row units (two 128-row MMAs sharing each B panel), for long-K products.
cudaError_t launch_gemm_tc(const GemmOperand& A, const GemmOperand& B, int M, int N, int splits, bool two_row_tiles,
                           const GemmEpi& e, int n_sms, int* d_err, cudaStream_t st, long long* launches);
// CTAs of that launch.
int gemm_tc_grid(int M, int N, int splits, bool two_row_tiles, int kext, int n_sms);

// Exponent e of the exact power-of-two scale 2^e that brings max |Z| of an
// instance into [2^13, 2^14) before the FP16 hi/lo split (the HERK epilogue
// multiplies by 2^-2e).
__device__ __forceinline__ int fp16_scale_exp(float amax) {
    if (!(amax > 0.f) || !(amax < 3.0e38f)) return 0;
    int e;
    frexpf(amax, &e);
    e = 14 - e;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

}  // namespace mv
