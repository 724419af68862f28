/*
 * matvis.h -- C-ABI of a single-GPU (sm_103a) matrix-based visibility
 * simulator after Kittiwisit et al., "matvis: a matrix-based visibility
 * simulator for fast forward modelling of many-element 21 cm arrays"
 * (arXiv:2312.09763).
 *
 * For every (time, frequency) instance the library runs Algorithm 2 of the
 * paper (Sec. 3.1) on the GPU:
 *   (i)   rotate the sources to East-North-Up with the FP64 matrix R(t) of
 *         eq. "rotation" (Sec. 2.3) and drop those with Up <= 0;
 *   (ii)  evaluate the beam of every unique antenna type at the live sources
 *         (analytic Gaussian, or a gridded beam interpolated as Sec. 2.4);
 *   (iii) form the per-antenna phase (nu/c) x_a . s_hat in FP64 and reduce it
 *         exactly modulo one turn;
 *   (iv)  build Z[(a,p),(s,k)] = sqrt(I_s) A^{pk}_{beta(a)}(s) exp(-2 pi i phase)
 *         (eq. "littlez"; Sec. 2.2);
 *   (v)   expand V = Z Z^dagger (eq. "zz") on the tensor cores (FP16 x3 split
 *         precision, FP32 accumulation) or on the CUDA cores (FP32).
 *
 * Conventions (all calls):
 *   - Every call returns an mv_status; no C++ exception crosses this ABI.
 *     On failure mv_last_error() describes the problem (thread-local string,
 *     valid until the next call on the same thread).
 *   - Input arrays are borrowed for the duration of the call and copied; the
 *     caller keeps ownership.  Output buffers are caller-owned.
 *   - A context is bound to one device and is not thread-safe.  Work is
 *     ordered on the stream given to mv_simulate (NULL = the context's own
 *     stream).
 *   - Angles are radians, lengths metres, frequencies Hz, fluxes Jy.
 *   - Output V for one instance is the full N x N Hermitian matrix,
 *     N = n_feed * n_ant, complex64 (interleaved re, im float), row-major,
 *     row/column index (a, p) = a * n_feed + p; V[a][b] = sum_s Z_a conj(Z_b),
 *     i.e. the baseline is b_ab = x_a - x_b (Sec. 2.2, fringe factorisation).
 */
#ifndef MATVIS_GB300_H
#define MATVIS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mv_ctx mv_ctx; /* opaque; owns all device state of one simulator */

typedef enum {
    MV_OK = 0,
    MV_ERR_ARG = 1,            /* invalid argument (size, range, NaN, negative flux, ...) */
    MV_ERR_OOM = 2,            /* device or host allocation failed */
    MV_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    MV_ERR_STATE = 4,          /* call out of order (e.g. simulate before set-up) */
    MV_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait gave up; results invalid */
    MV_ERR_UNSUPPORTED = 6     /* feature not available on this device / build */
} mv_status;

/* Arithmetic of steps (iv)-(v).  Both modes meet max |V - V_oracle| /
 * max |V_oracle| <= 1e-5 against the FP64 definition.  Value 1 is not used:
 * a split into two BF16 pieces keeps only 16 significant bits of each entry of
 * Z (representation error up to 2^-16 = 1.5e-5 relative per entry), which
 * cannot meet that bound, so no BF16 mode is offered (MV_ERR_ARG). */
typedef enum {
    MV_PREC_FP32 = 0,   /* Z and V = Z Z^H in FP32 on CUDA cores */
    MV_PREC_FP16X3 = 2  /* Z scaled by an exact power of two (one per group of channels of one
                           time) into FP16 range and split as hi + lo FP16 (11 significant bits
                           each, 22 together); hi hi^T + hi lo^T + lo hi^T on tcgen05 with FP32
                           accumulation: the matrix product of step (v) in split precision */
} mv_precision;

typedef enum {
    MV_INTERP_CUBIC = 0,    /* Keys cubic convolution in az, za and frequency */
    MV_INTERP_BILINEAR = 1  /* linear in az and za, Keys cubic in frequency */
} mv_interp;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer or NULL; both run on the host thread that called
 * into the library, outside any kernel. */
typedef struct {
    void *(*alloc)(size_t bytes, int device, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, int device, void *stream, void *user);
    void *user;
} mv_allocator;

typedef struct {
    int interp;                 /* mv_interp for gridded beams (default cubic) */
    int max_batch;              /* channels of one time processed per launch (0 = auto, at most 256) */
    int herk_flush_kblocks;     /* tensor-core HERK: 64-column k-blocks accumulated in one
                                   TMEM buffer before it is added into the FP32 running
                                   sum (0 = auto = 4) */
    int herk_split;             /* split of the source axis across CTAs (0 = auto) */
    mv_allocator allocator;     /* alloc == NULL: cudaMalloc / cudaFree */
    int herk_tile_n;            /* tensor-core HERK tile width: 128 or 256 columns (0 = auto) */
    int use_graph;              /* capture each call shape's launch sequence in a CUDA graph and
                                   replay it (default 1; calls with kernel timing run uncaptured) */
    int overlap_batches;        /* 1: with two or more batches, build the Z matrices of one batch
                                   on a second stream while the HERK of the previous one runs (two
                                   workspace sets); 0 (default): one set, strictly in order */
    int fuse_zbuild;            /* 1 (default): with two or more batches and a tensor-core
                                   precision, the HERK launch of batch b also builds the Z matrices
                                   of batch b + 1 on extra warps of every SM (two workspace sets;
                                   one feed and one axis, or two and two), unless mv_autotune timed
                                   separate launches faster for the call's shape; 0: the Z build
                                   runs as its own launch.  Takes precedence over overlap_batches. */
} mv_options;

/* A tensor-core HERK configuration chosen by mv_autotune. */
typedef struct {
    int tile_n;          /* 128 or 256 */
    int split;           /* source-axis split */
    int flush_kblocks;   /* 64-source k-blocks per TMEM flush */
    int candidates;      /* configurations timed */
    double herk_ms;      /* best time of one batch: the HERK launch (with the next batch's Z build when
                            fused), or the HERK and the batch's own Z-side launches */
    int fused;           /* 1: the HERK launch of a batch builds the next batch's Z planes;
                            0: every batch's Z build runs as its own launches */
} mv_tuning;

/* Fill *opt with defaults. */
void mv_default_options(mv_options *opt);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * Fails with MV_ERR_UNSUPPORTED unless the device is compute capability 10.3. */
mv_status mv_create(mv_ctx **out, int device, const mv_options *opt);

/* Release every device buffer of the context.  NULL is accepted. */
void mv_destroy(mv_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *mv_last_error(void);

/* Sky model (Sec. 3.1 inputs: X_eq from eq. "xeq", intensities I >= 0).
 * ra, dec: [n_src] radians.  flux_ref: [n_src] Jy at nu_ref, finite and >= 0
 * (the paper requires a positive intensity vector).  spec_idx: [n_src]
 * spectral indices alpha (NULL = 0), I_s(nu) = flux_ref_s (nu / nu_ref)^alpha_s.
 * n_src >= 1.  Host pointers; copied. */
mv_status mv_init_sky(mv_ctx *ctx, int64_t n_src, const double *ra, const double *dec,
                      const double *flux_ref, const double *spec_idx, double nu_ref);

/* Perturbed source coordinates of Algorithm 1 (Sec. 2.3, the "fast"
 * coordinate scheme), steps (ii) and (iv)-(vi); host only (no context, no
 * device).  The rigid rotation of eq. "rotation" lacks the time-dependent
 * astrometric corrections; this call moves each source to fictitious
 * equatorial coordinates (RA', Dec') for which the rigid rotation at the
 * reference LST gives exactly the caller's apparent direction:
 *   X_hrz = (cos alt sin az, cos alt cos az, sin alt)   (East, North, Up),
 *   X_eq' = R(lst_ref)^T X_hrz                          (R^-1 = R^T),
 *   RA' = atan2(y, x) in [0, 2 pi), Dec' = atan2(z, sqrt(x^2 + y^2)).
 * Steps (i) and (iii) -- the apparent LST at the reference time and the
 * apparent (alt, az) of every source then -- are the caller's (the paper uses
 * astropy).  Pass (RA', Dec') to mv_init_sky; for long runs cut the times into
 * chunks, each with its own reference time, perturbed catalogue and
 * mv_init_sky (the correction degrades away from t_ref).
 * alt_rad, az_rad: [n_src] radians, az from North through East, |alt| <= pi/2;
 * lst_ref_rad: apparent LST at the reference time; latitude_rad: |lat| <= pi/2.
 * ra_out, dec_out: [n_src] radians.  Host pointers (caller-owned).
 * MV_ERR_ARG for n_src < 1, NULL pointers or non-finite / out-of-range
 * angles (the message names the first bad source). */
mv_status mv_perturb_sky(int64_t n_src, const double *alt_rad, const double *az_rad, double lst_ref_rad,
                         double latitude_rad, double *ra_out, double *dec_out);

/* Fully polarised sky (Sec. 2.1 coherency, Sec. 2.2 eq. "fullz"): Stokes Q,
 * U, V of every source of the last mv_init_sky, in Jy at nu_ref, host
 * arrays of n_src (copied).  The coherency in the beam's (theta, phi)
 * component basis is C = [[I + Q, U + iV], [U - iV, I - Q]], static in
 * celestial coordinates as in the paper, and all four Stokes follow the
 * source's power law.  Z becomes sum_k A^{pk} F M_{kk''} with M the
 * lower-triangular Cholesky factor of C (formed in FP64 on the host), so V
 * stays Z Z^dagger.  Needs Q^2 + U^2 + V^2 <= I^2 (1 + 1e-6) per source
 * (MV_ERR_ARG otherwise) and, at simulate time, a two-axis gridded beam or a
 * surrogate of one (MV_ERR_STATE otherwise).  q = u = v = NULL returns to an
 * unpolarised sky; a later mv_init_sky also does. */
mv_status mv_set_sky_polarisation(mv_ctx *ctx, int64_t n_src, const double *stokes_q,
                                  const double *stokes_u, const double *stokes_v);

/* Analytic unpolarised Gaussian E-field beam, the same for every antenna:
 * A(za) = exp(-4 ln2 za^2 / fwhm^2) (Sec. 2.4 analytic beams).  fwhm > 0. */
mv_status mv_set_beam_gaussian(mv_ctx *ctx, double fwhm_rad);

/* Gridded beams (Sec. 2.4): values complex64 [n_beam][n_feed][n_ax][n_nu][n_za][n_az]
 * (interleaved re, im), az-fastest.  Axes: nu_m = nu0 + m dnu, za_i = i dza
 * (the zenith is the grid's pole, row 0), az_j = j daz with n_az * daz = 2 pi
 * (periodic; n_az even).  n_feed, n_ax in {1, 2}; n_ax = 2 means the columns
 * are (theta, phi) E-field components, which change sign across the pole.
 * Interpolation per mv_options.interp.  Rows past the last za node repeat the
 * last row.  Host pointer; copied.
 * The grid's first za row is always the zenith (no za0 argument): Sec. 2.4
 * needs the zenith treated as the grid's pole, and the pole reflection (a
 * stencil row at za < 0 is row -za at az + pi) is only defined when row 0 sits
 * on it. */
mv_status mv_set_beam_grid(mv_ctx *ctx, int n_beam, int n_feed, int n_ax, int n_nu, int n_za,
                           int n_az, const float *values_c64, double nu0, double dnu,
                           double dza, double daz);

/* Antenna layout (Sec. 3.1 inputs D and a_i): enu [n_ant][3] East-North-Up
 * metres; beam_idx [n_ant] index of each antenna's unique beam (NULL = all
 * 0); latitude of the array.  Host pointers; copied. */
mv_status mv_set_antennas(mv_ctx *ctx, int n_ant, const double *enu, const int32_t *beam_idx,
                          double latitude_rad);

/* Simulate n_t x n_nu instances (Algorithm 2 for every LST and frequency).
 * lst: [n_t] local sidereal times (radians; they define R(t), Sec. 3.1);
 * nu: [n_nu] Hz, inside the beam grid's cubic margin for gridded beams.
 * V: complex64 [n_t][n_nu][N][N]; a device pointer if V_on_device, else host
 * memory written before the call returns.  stream: cudaStream_t or NULL.
 * With V on the device the call returns once the work is queued; device-side
 * wait timeouts are reported by mv_check_device_status. */
mv_status mv_simulate(mv_ctx *ctx, int n_t, const double *lst, int n_nu, const double *nu,
                      mv_precision prec, void *V, int V_on_device, void *stream);

/* Simulate an explicit list of (lst, nu) pairs: V complex64 [n_pairs][N][N].
 * Every (time, frequency) instance of Algorithm 2 is independent (Sec. 3.1:
 * frequency is the outer loop and times the inner one, with no interaction
 * between them), so an arbitrary list of instances is as valid a call as the
 * n_t x n_nu grid of mv_simulate; lst[i], nu[i] as there.  Arguments, output
 * placement, stream and errors as mv_simulate. */
mv_status mv_simulate_pairs(mv_ctx *ctx, int n_pairs, const double *lst, const double *nu,
                            mv_precision prec, void *V, int V_on_device, void *stream);

/* Autotune the tensor-core HERK for calls shaped like this one (the paper
 * leaves the matrix-product kernel to cuBLAS, Sec. 4.3; here it is the
 * project's own and its tile width, source-axis split and flush interval are
 * tuned).  Runs the first batch of the call (mv_simulate's plan, or
 * mv_simulate_pairs' plan if pairs != 0 with n_t == n_nu pairs), times the
 * HERK of that batch under each candidate (tile width 128 or 256 -- 128 only
 * when the Z build is fused, and then every trial also builds a batch of Z
 * planes --, split of the source axis 1 to 64, flush every 4, 8 or 16
 * k-blocks) with CUDA events on the context's stream, and keeps the fastest
 * for later calls with the same matrix size, batch size and precision.
 * Synchronises.  prec must be a tensor-core precision.  out may be NULL. */
mv_status mv_autotune(mv_ctx *ctx, int n_t, const double *lst, int n_nu, const double *nu,
                      mv_precision prec, int pairs, mv_tuning *out);

/* Synchronise the context's work and report (and clear) a device-side error
 * flag (MV_ERR_DEVICE_TIMEOUT) or a pending CUDA error.  The paper has no
 * counterpart (its GPU steps are synchronous library calls); here every
 * bounded wait of the tensor-core kernels reports through this flag. */
mv_status mv_check_device_status(mv_ctx *ctx, void *stream);

/* Self-test of the failure path: launches one thread that waits, with the
 * bounded mbarrier wait every tensor-core kernel uses but a limit of limit_s
 * (0 < limit_s <= 10), on a barrier nothing completes.  The kernel gives up,
 * records the timeout and returns; the call synchronises and returns what
 * mv_check_device_status reports, MV_ERR_DEVICE_TIMEOUT, leaving the context
 * usable (no fault, no hang). */
mv_status mv_selftest_wait_timeout(mv_ctx *ctx, double limit_s);

/* Number of live (Up > 0) sources at each LST, as the last mv_simulate or
 * mv_simulate_pairs call computed them on the device (its instances, in
 * order): out [n] int64.  Synchronises. */
mv_status mv_last_live_counts(mv_ctx *ctx, int n, int64_t *out);

/* Number of kernel launches the last simulate call issued. */
int64_t mv_last_launch_count(mv_ctx *ctx);

/* Kernel timing (the paper profiles each step of Algorithm 2 separately,
 * Sec. 4.1).  When enabled, every launch is bracketed by two CUDA events
 * recorded on the stream it is launched on; counters accumulate across
 * simulate calls until the next mv_profile_enable.  Kinds follow the steps
 * of Algorithm 2. */
typedef enum {
    MV_KERNEL_CULL = 0,    /* step (i): rotation, horizon cut, compaction */
    MV_KERNEL_BEAM = 1,    /* step (ii): beam planes and beam x sqrt(I) at live sources */
    MV_KERNEL_ZBUILD = 2,  /* steps (iii)-(iv): FP64 phase, Z */
    MV_KERNEL_HERK = 3,    /* step (v): V = Z Z^dagger */
    MV_KERNEL_KINDS = 4
} mv_kernel_kind;

/* ------------------------------------------------------------- redundancy
 * Baseline redundancy (Appendix A of the paper, "Utilising baseline
 * redundancies").  Baselines (a, b), a <= b, whose vectors x_a - x_b agree on a
 * tol_m grid (each component rounded to a multiple of tol_m) and whose beams
 * agree have equal visibilities; a baseline whose vector is the reverse of
 * another's (beams swapped) has the conjugate visibility.  Each group has one
 * representative, its first member in lexicographic order; groups are
 * numbered in the order of their representatives.
 *
 * mv_redundancy_plan (host only: no context, no device) groups the baselines
 * of n_ant antennas (enu [n_ant][3] metres, beam_idx [n_ant] or NULL = all 0)
 * and plans the cover of the representatives the HERK computes: Appendix A's
 * sub-matrix heuristic (first antennas sorted by multiplicity, cut into 1-3
 * slices at a density threshold), in both orientations, each sub-matrix a block
 * of contiguous rows and columns of V in a permuted antenna order, costed in
 * 128-row x tile_n-column (128 or 256) tiles of the 2 n_feed-row real Gram
 * matrix; the whole lower triangle is kept when no cover is cheaper.
 * Outputs (each may be NULL; sizes: n_bl = n_ant (n_ant + 1) / 2):
 *   n_unique          number of groups
 *   rep_a, rep_b      [n_bl] (only the first n_unique written) representatives
 *   group_of          [n_bl] group of baseline (a, b), a <= b, row-major over a then b
 *   conj_of           [n_bl] 1 where (a, b) is a reversed baseline of its group:
 *                     V_ab^{pq} = conj(V_rep^{qp}) (feeds swapped), else V_ab = V_rep
 *   perm              [n_ant] position of antenna a in the cover's order
 *   kind              0 whole triangle, 1 blocks hold (rep_a, rep_b) as (row, column),
 *                     2 as (rep_b, rep_a)
 *   n_blocks, blocks  [4][4] int32: row0, row1, col0, col1 (positions) per block
 *   tiles             [2]: tiles of the chosen cover, tiles of the whole triangle
 * MV_ERR_ARG for bad sizes, non-finite positions, tol_m <= 0 or n_feed < 1. */
mv_status mv_redundancy_plan(int n_ant, const double *enu, const int32_t *beam_idx, double tol_m, int n_feed,
                             int tile_n, int64_t *n_unique, int32_t *rep_a, int32_t *rep_b, int32_t *group_of,
                             int8_t *conj_of, int32_t *perm, int32_t *kind, int32_t *n_blocks, int32_t *blocks,
                             int64_t *tiles);

/* Plan the redundant-group output for the context's antennas and beam (as
 * mv_redundancy_plan with tile_n = 128): the Z planes of mv_simulate_unique
 * are then built in the cover's antenna order and the HERK computes only the
 * tiles of the cover.  tol_m <= 0 turns it off.  *n_unique (may be NULL)
 * receives the number of groups.  MV_ERR_STATE before set_antennas and a
 * beam; a later set_antennas (or a beam with another feed count) drops the
 * plan. */
mv_status mv_set_redundancy(mv_ctx *ctx, double tol_m, int64_t *n_unique);

/* As mv_simulate, but one value per redundant group: V [n_t][n_nu][n_unique]
 * [n_feed][n_feed] complex64, entry [g][p][q] = V^{pq} of the group's
 * representative (rep_a, rep_b) of mv_redundancy_plan (every baseline of the
 * group has this value, or where conj_of says so V_ab^{pq} = conj(V^{qp})).  Needs
 * mv_set_redundancy and a tensor-core precision (MV_ERR_ARG for FP32). */
mv_status mv_simulate_unique(mv_ctx *ctx, int n_t, const double *lst, int n_nu, const double *nu,
                             mv_precision prec, void *V, int V_on_device, void *stream);

/* Rotation and horizon cut of one LST without any device allocation.
 *
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they run this step -- hosts whose device memory all
 * belongs to a framework's own pool (a cudaMalloc beside it can fail or
 * fragment it), and latency-critical loops that cannot take cudaMalloc's
 * implicit device synchronisation.  It runs the same kernels as step (i) of
 * mv_simulate, but their scratch (per-block live counts and offsets, and the
 * 3 x 3 rotation) lives in a static device array of 64 KB that every GPU
 * loading this library holds until the process exits.  The rotation reaches
 * the device as a kernel argument, so no host buffer outlives the call.
 *
 * Limits and sharing: 1 <= n_src <= 2,097,152 and |latitude_rad| <= pi/2,
 * else MV_ERR_ARG.  Every call
 * on a device shares that array; calls that overlap on the GPU (for example
 * on two unsynchronised streams) race and give wrong results.  Nothing in it
 * needs clearing: a call writes every entry it reads.  The first call on each
 * device resolves the array's device address with cudaGetSymbolAddress on the
 * current device (once per device, under a lock).
 *
 * Arguments (device pointers unless stated): xeq_dev [3][n_src] FP64 SoA
 * (x, y, z of eq. "xeq"); lst_rad, latitude_rad host values; outputs, for the
 * live sources (Up > 0) in catalogue order: live_idx_dev [n_src] int32
 * catalogue indices, enu_dev [3][n_src] FP64 SoA (East, North, Up),
 * azza_dev [n_src][2] FP32 (az, za; 8-byte aligned), n_live_dev [1] int32.
 * Entries past n_live are left untouched.  Runs on the current device and on
 * `stream` (NULL = legacy default stream); returns once the work is queued.
 * Errors go to mv_last_error(). */
mv_status mv_horizon_cull_static(int64_t n_src, const double *xeq_dev, double lst_rad, double latitude_rad,
                                 int32_t *live_idx_dev, double *enu_dev, float *azza_dev,
                                 int32_t *n_live_dev, void *stream);

/* ---------------------------------------------------------------------
 * Learned beam.  (The calls are named mv_surrogate_*: create, train, params,
 * set_params, eval, grad, save, load; training reports its first and last
 * loss through mv_surrogate_train's arguments rather than a report struct, and
 * mv_mlp_config is the network's configuration.)  The paper interpolates
 * gridded beams (Sec. 2.4) and notes
 * that per-antenna beams make that step expensive (Sec. 3.1); here a
 * Fourier-feature MLP stands in for a set of gridded beams:
 *   x = (az / 2 pi, za / (pi/2), (nu - nu_mid) / nu_half), nu_mid and nu_half
 *       the centre and half-width of the grid's frequency range;
 *   f = [sin(2 pi B x), cos(2 pi B x), e_beta]  (B: n_freq x 3 fixed, az column
 *       integer so az stays periodic; e_beta the learned embedding of beam beta);
 *   h_l = relu(W_l h_{l-1} + b_l) for depth hidden layers of `width` units;
 *   y = W_out h + b_out: 2 n_feed n_ax real outputs (re, im of each component
 *       in (feed, axis) order).
 * It is trained on the GPU (every product of the forward and backward pass on
 * the tcgen05 tensor cores with BF16 operands and FP32 accumulation, FP32
 * master weights, Adam, MSE) on samples (beta, az, za, nu) drawn uniformly and
 * labelled by the Keys interpolation of the gridded beam set with
 * mv_set_beam_grid, one embedding per gridded beam.  The first layer's input
 * is padded to d0p = max(64, 2 n_freq + emb_dim rounded up to 32) columns. */
typedef struct {
    int n_freq;                          /* Fourier frequencies (default 64) */
    int emb_dim;                         /* embedding size (16); 2 n_freq + emb_dim <= 240 */
    int width;                           /* hidden width (256; a multiple of 16 in [64, 256]) */
    int depth;                           /* hidden layers (4; 1 to 16) */
    float sigma_az, sigma_za, sigma_nu;  /* scales of B's columns (2, 3, 1) */
    uint64_t seed;                       /* initial weights and B */
} mv_mlp_config;

void mv_default_mlp_config(mv_mlp_config *cfg);

/* Create (or replace) the surrogate for the current gridded beams.  cfg may be
 * NULL (defaults).  MV_ERR_STATE without a gridded beam. */
mv_status mv_surrogate_create(mv_ctx *ctx, const mv_mlp_config *cfg);

/* Train for `steps` Adam steps of `batch` samples (batch a multiple of 8), the
 * learning rate following a cosine from lr0 to lr1; sample draws use `seed`
 * (step i draws the batch of counter i: beams stratified over the batch,
 * (az, za, nu) uniform, targets the gridded beams' Keys-cubic interpolation).
 * loss_first / loss_last (may be NULL) receive the MSE of the first and last
 * step.  The first call for a batch size with enough steps (12; 15 when the
 * batch takes more than four rounds of 128-row tiles on the SMs) times three
 * or four splits of the SMs between the training launches and the sampler of
 * the next step (which runs beside them) over its first steps and keeps the
 * fastest for that batch size.  Synchronises. */
mv_status mv_surrogate_train(mv_ctx *ctx, int steps, int batch, float lr0, float lr1, uint64_t seed,
                             double *loss_first, double *loss_last);

/* Parameters: *n_params receives the count; if host != NULL the FP32 master
 * vector is copied there; if fourier != NULL, B ([n_freq][3]); if layout !=
 * NULL, 2 (depth + 1) + 2 offsets: W_l, b_l for l = 0..depth (W_depth is the
 * output layer, stored [8][width]; W_0 is [width][d0p] with d0p = max(64,
 * 2 n_freq + emb_dim rounded up to 32)), then the embedding offset and d0p. */
mv_status mv_surrogate_params(mv_ctx *ctx, int64_t *n_params, float *host, float *fourier, int64_t *layout);
mv_status mv_surrogate_set_params(mv_ctx *ctx, const float *host);

/* Evaluate at n points (host arrays): out [n][2 n_feed n_ax] host. */
mv_status mv_surrogate_eval(mv_ctx *ctx, int n, const int32_t *beam, const double *az, const double *za,
                            const double *nu, float *out);

/* Loss and gradient of all parameters for n given samples and targets
 * ([n][2 n_feed n_ax]); grads [n_params] host, no update.  n a multiple of 8. */
mv_status mv_surrogate_grad(mv_ctx *ctx, int n, const int32_t *beam, const double *az, const double *za,
                            const double *nu, const float *target, float *grads, double *loss);

/* Save / load the surrogate (configuration, B and parameters) to a file. */
mv_status mv_surrogate_save(mv_ctx *ctx, const char *path);
mv_status mv_surrogate_load(mv_ctx *ctx, const char *path);

/* enable != 0: mv_simulate evaluates the beams with the surrogate (antenna a
 * uses embedding beam_idx[a]) instead of interpolating the grid. */
mv_status mv_set_beam_surrogate(mv_ctx *ctx, int enable);

/* Device memory of the two beam models (the cost Sec. 3.1 names for
 * per-antenna beams): *grid_bytes, the gridded beams as held (all unique
 * beams' grids plus the per-channel planes of the last call; 0 without a
 * gridded beam); *surrogate_bytes, what evaluating the surrogate reads (FP32
 * parameters, their BF16 copy, the Fourier matrix; 0 without a surrogate).
 * Either pointer may be NULL. */
mv_status mv_beam_model_bytes(mv_ctx *ctx, int64_t *grid_bytes, int64_t *surrogate_bytes);

/* enable != 0 switches timing on and clears the counters; 0 switches it off. */
mv_status mv_profile_enable(mv_ctx *ctx, int enable);

/* Synchronise and read the counters of one kind: number of launches and the
 * sum of their event-measured durations in milliseconds. */
mv_status mv_profile_read(mv_ctx *ctx, int kind, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* MATVIS_GB300_H */
