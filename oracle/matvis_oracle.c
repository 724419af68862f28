/*
 * matvis_oracle.c -- plain, slow, FP64 CPU reference for the matvis visibility
 * simulator (Kittiwisit et al., "matvis: a matrix-based visibility simulator",
 * arXiv:2312.09763).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * constant table or helper with the CUDA library, and it never calls it.
 *
 * What it computes is the plain definition, evaluated per baseline:
 *
 *   V_ab^{pq}(t, nu) = sum_{s : Up_s(t) > 0}  I_s(nu)
 *                        * sum_k A_{beta(a)}^{pk}(nu, s) conj(A_{beta(b)}^{qk}(nu, s))
 *                        * exp(-2 pi i (nu / c) (x_a - x_b) . X_hrz,s(t))
 *
 * which is the discrete RIME of Sec. 2.1 (eq. "matvisrime") with the delay of
 * eq. "matvisdelay" and an unpolarised coherency C = I * identity (Sec. 2.2,
 * the case that leads to eq. "littlez").  Source directions follow eq. "xeq"
 * and eq. "rotation" (Sec. 2.3); beams follow Sec. 2.4.  Every floating-point
 * step is IEEE double.  Compile with -ffp-contract=off so that no product is
 * fused into an add behind our back (the horizon test Up > 0 must be taken on
 * exactly the value written below).
 *
 * Readings of the paper that this file fixes (the paper leaves them open):
 *   - eq. "rotation" is used with H = -LST, so a source with RA = LST and
 *     Dec = latitude lands at the zenith (0, 0, 1) of the East-North-Up frame.
 *   - live sources are those with Up > 0 strictly.
 *   - azimuth az = atan2(East, North) in [0, 2 pi) (North through East),
 *     zenith angle za = acos(Up).
 *   - the Gaussian analytic beam is the E-field amplitude
 *     A(za) = exp(-4 ln2 za^2 / FWHM^2).
 *   - gridded beams are interpolated with the Keys (1981) cubic-convolution
 *     kernel (a = -1/2) separably in az, za and frequency ("cubic"), or with
 *     linear weights in az and za and the Keys kernel in frequency
 *     ("bilinear"); az is periodic; a stencil row at negative za is the row
 *     at +za on the opposite azimuth (az + pi), negated for two-axis (theta,
 *     phi) E-field components and unchanged for single-axis beams; rows past
 *     the last za node take the last row.
 *   - I_s(nu) = S_s (nu / nu_ref)^alpha_s.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C_LIGHT 299792458.0 /* speed of light, m/s */
#define ORC_PI 3.14159265358979323846264338327950288

/* Problem description shared with the Python wrapper (ctypes mirror). */
typedef struct {
    /* sky */
    int64_t n_src;
    const double *ra, *dec;      /* radians */
    const double *flux_ref;      /* Jy at nu_ref, >= 0 */
    const double *spec_idx;      /* may be NULL (all zero) */
    double nu_ref;               /* Hz */
    /* array */
    int32_t n_ant;
    const double *enu;           /* [n_ant][3] metres */
    const int32_t *beam_idx;     /* may be NULL (all zero) */
    double lat;                  /* radians */
    /* beam */
    int32_t beam_kind;           /* 0 uniform, 1 gaussian, 2 grid, 3 tabulated (see inst_prepare) */
    double fwhm;                 /* radians (gaussian) */
    int32_t n_beam, n_feed, n_ax;
    int32_t n_nu, n_za, n_az;
    const double *grid;          /* complex128 [beam][feed][ax][nu][za][az] */
    double nu0, dnu, dza, daz;   /* grid axes: nu_m = nu0 + m dnu, za_i = i dza, az_j = j daz */
    int32_t interp;              /* 0 cubic (Keys), 1 bilinear in az/za */
} orc_problem;

/* ---------------------------------------------------------------- coords */

/* eq. "xeq" (Sec. 2.3): Cartesian equatorial unit vector of each source. */
void orc_xeq(int64_t n, const double *ra, const double *dec, double *xyz)
{
    for (int64_t s = 0; s < n; ++s) {
        double cd = cos(dec[s]);
        xyz[3 * s + 0] = cos(ra[s]) * cd;
        xyz[3 * s + 1] = sin(ra[s]) * cd;
        xyz[3 * s + 2] = sin(dec[s]);
    }
}

/* eq. "rotation" (Sec. 2.3), row-major, with hour angle H = -LST and
 * latitude l.  Rows are East, North, Up. */
void orc_rotation(double lst, double lat, double *R)
{
    double H = -lst;
    double sH = sin(H), cH = cos(H), sl = sin(lat), cl = cos(lat);
    R[0] = sH;       R[1] = cH;       R[2] = 0.0;
    R[3] = -sl * cH; R[4] = sl * sH;  R[5] = cl;
    R[6] = cl * cH;  R[7] = -cl * sH; R[8] = sl;
}

/* X_hrz = R X_eq (Sec. 2.3), each component as (R_i0 x + R_i1 y) + R_i2 z. */
void orc_to_topo(const double *R, int64_t n, const double *xyz, double *enu)
{
    for (int64_t s = 0; s < n; ++s) {
        double x = xyz[3 * s], y = xyz[3 * s + 1], z = xyz[3 * s + 2];
        for (int i = 0; i < 3; ++i) {
            double p0 = R[3 * i] * x;
            double p1 = R[3 * i + 1] * y;
            double p2 = R[3 * i + 2] * z;
            enu[3 * s + i] = (p0 + p1) + p2;
        }
    }
}

/* Azimuth (N through E, [0, 2 pi)) and zenith angle of an ENU unit vector. */
void orc_azza(int64_t n, const double *enu, double *az, double *za)
{
    for (int64_t s = 0; s < n; ++s) {
        double e = enu[3 * s], no = enu[3 * s + 1], u = enu[3 * s + 2];
        double a = atan2(e, no);
        if (a < 0.0) a += 2.0 * ORC_PI;
        if (u > 1.0) u = 1.0;
        if (u < -1.0) u = -1.0;
        az[s] = a;
        za[s] = acos(u);
    }
}

/* ------------------------------------------------------------------ beams */

/* Keys (1981) cubic-convolution kernel with a = -1/2. */
double orc_keys(double x)
{
    const double a = -0.5;
    double t = fabs(x);
    if (t <= 1.0) return ((a + 2.0) * t - (a + 3.0)) * t * t + 1.0;
    if (t < 2.0) return ((a * t - 5.0 * a) * t + 8.0 * a) * t - 4.0 * a;
    return 0.0;
}

/* Stencil of a regular axis at coordinate u (in node units): first node and
 * weights.  Cubic: 4 nodes floor(u)-1 .. floor(u)+2.  Linear: 2 nodes. */
static int stencil(double u, int cubic, int *first, double *w)
{
    double f = floor(u);
    double t = u - f;
    if (cubic) {
        *first = (int)f - 1;
        w[0] = orc_keys(t + 1.0);
        w[1] = orc_keys(t);
        w[2] = orc_keys(1.0 - t);
        w[3] = orc_keys(2.0 - t);
        return 4;
    }
    *first = (int)f;
    w[0] = 1.0 - t;
    w[1] = t;
    return 2;
}

/* Gridded beam component (beam b, feed p, axis k) at (az, za, nu), Sec. 2.4.
 * Returns 0, or -1 if nu is outside the grid's cubic margin. */
int orc_beam_grid_eval(const orc_problem *P, int b, int p, int k,
                       double az, double za, double nu, double *re, double *im)
{
    int nf, nz, na = P->n_az;
    double wf[4], wz[4], wa[4];
    int f0, z0, a0;
    int nwf = stencil((nu - P->nu0) / P->dnu, 1, &f0, wf);
    if (f0 < 0 || f0 + nwf - 1 > P->n_nu - 1) return -1;
    int cubic = (P->interp == 0);
    int nwz = stencil(za / P->dza, cubic, &z0, wz);
    int nwa = stencil(az / P->daz, cubic, &a0, wa);
    double pole_sign = (P->n_ax == 2) ? -1.0 : 1.0;
    const double *base = P->grid
        + 2 * (int64_t)(((int64_t)b * P->n_feed + p) * P->n_ax + k) * P->n_nu * P->n_za * P->n_az;
    double sr = 0.0, si = 0.0;
    for (nf = 0; nf < nwf; ++nf) {
        const double *plane = base + 2 * (int64_t)(f0 + nf) * P->n_za * P->n_az;
        for (nz = 0; nz < nwz; ++nz) {
            int row = z0 + nz;
            int shift = 0;
            double sgn = 1.0;
            if (row < 0) { row = -row; shift = na / 2; sgn = pole_sign; }
            if (row > P->n_za - 1) row = P->n_za - 1;
            double wzf = wf[nf] * wz[nz] * sgn;
            for (int m = 0; m < nwa; ++m) {
                int col = ((a0 + m + shift) % na + na) % na;
                const double *v = plane + 2 * ((int64_t)row * na + col);
                sr += wzf * wa[m] * v[0];
                si += wzf * wa[m] * v[1];
            }
        }
    }
    *re = sr;
    *im = si;
    return 0;
}

/* Beam component of beam b (feed p, axis k) at one direction. */
static int beam_eval(const orc_problem *P, int b, int p, int k,
                     double az, double za, double nu, double *re, double *im)
{
    if (P->beam_kind == 0) { *re = 1.0; *im = 0.0; return 0; }
    if (P->beam_kind == 1) {
        *re = exp(-4.0 * log(2.0) * za * za / (P->fwhm * P->fwhm));
        *im = 0.0;
        return 0;
    }
    return orc_beam_grid_eval(P, b, p, k, az, za, nu, re, im);
}

/* Evaluate beam components for a list of directions: out complex128
 * [beam][feed][ax][n]. */
int orc_beam_eval_many(const orc_problem *P, int64_t n, const double *az,
                       const double *za, double nu, double *out)
{
    int nb = P->beam_kind >= 2 ? P->n_beam : 1;
    for (int b = 0; b < nb; ++b)
        for (int p = 0; p < P->n_feed; ++p)
            for (int k = 0; k < P->n_ax; ++k)
                for (int64_t s = 0; s < n; ++s) {
                    int64_t o = (((int64_t)b * P->n_feed + p) * P->n_ax + k) * n + s;
                    if (beam_eval(P, b, p, k, az[s], za[s], nu, &out[2 * o], &out[2 * o + 1]))
                        return -1;
                }
    return 0;
}

/* ------------------------------------------------------------- instance */

typedef struct {
    int64_t n_live;
    double *enu;    /* [n_live][3] */
    double *flux;   /* [n_live] I_s(nu) */
    double *A;      /* complex128 [n_beam][feed][ax][n_live] */
    int64_t *idx;   /* [n_live] catalogue index */
} orc_inst;

static void inst_free(orc_inst *I)
{
    free(I->enu); free(I->flux); free(I->A); free(I->idx);
    memset(I, 0, sizeof(*I));
}

/* Steps (i)-(ii) of Algorithm 2 and the per-channel flux: rotate, cut at the
 * horizon, evaluate the beams of the live sources. */
static int inst_prepare(const orc_problem *P, double lst, double nu, orc_inst *I)
{
    int64_t n = P->n_src;
    double R[9];
    double *xyz = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *enu = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    memset(I, 0, sizeof(*I));
    orc_xeq(n, P->ra, P->dec, xyz);
    orc_rotation(lst, P->lat, R);
    orc_to_topo(R, n, xyz, enu);
    int64_t m = 0;
    for (int64_t s = 0; s < n; ++s)
        if (enu[3 * s + 2] > 0.0) ++m;
    int nb = P->beam_kind >= 2 ? P->n_beam : 1;
    int64_t mm = m > 0 ? m : 1;
    I->n_live = m;
    I->enu = malloc(sizeof(double) * 3 * mm);
    I->flux = malloc(sizeof(double) * mm);
    I->idx = malloc(sizeof(int64_t) * mm);
    I->A = malloc(sizeof(double) * 2 * (size_t)nb * P->n_feed * P->n_ax * mm);
    double *az = malloc(sizeof(double) * mm), *za = malloc(sizeof(double) * mm);
    int64_t j = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (!(enu[3 * s + 2] > 0.0)) continue;
        memcpy(&I->enu[3 * j], &enu[3 * s], 3 * sizeof(double));
        double alpha = P->spec_idx ? P->spec_idx[s] : 0.0;
        I->flux[j] = P->flux_ref[s] * pow(nu / P->nu_ref, alpha);
        I->idx[j] = s;
        ++j;
    }
    orc_azza(m, I->enu, az, za);
    int rc = 0;
    if (P->beam_kind == 3) {
        /* tabulated: P->grid holds complex128 [beam][feed][ax][m] for the live
         * sources in catalogue order (a caller-evaluated beam model) */
        memcpy(I->A, P->grid, sizeof(double) * 2 * (size_t)nb * P->n_feed * P->n_ax * (size_t)m);
    } else {
        rc = orc_beam_eval_many(P, m, az, za, nu, I->A);
    }
    free(az); free(za); free(xyz); free(enu);
    if (rc) inst_free(I);
    return rc;
}

/* Number of live sources (Up > 0) at one LST; -1 on bad input. */
int64_t orc_count_live(const orc_problem *P, double lst)
{
    int64_t n = P->n_src, m = 0;
    double R[9];
    double *xyz = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *enu = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    orc_xeq(n, P->ra, P->dec, xyz);
    orc_rotation(lst, P->lat, R);
    orc_to_topo(R, n, xyz, enu);
    for (int64_t s = 0; s < n; ++s)
        if (enu[3 * s + 2] > 0.0) ++m;
    free(xyz); free(enu);
    return m;
}

/* Direct per-baseline sum (eq. "matvisrime" with eq. "matvisdelay").
 * pairs: n_pairs (a, b) antenna pairs (pa[i], pb[i]); out complex128
 * [n_pairs][n_feed][n_feed].  If n_pairs < 0 all N x N entries are computed
 * into out[(a n_feed + p)][(b n_feed + q)] with N = n_feed n_ant.
 * Returns 0, -1 (frequency outside the beam grid) or -2 (bad index). */
int orc_vis(const orc_problem *P, double lst, double nu, int64_t n_pairs,
            const int32_t *pa, const int32_t *pb, double *out, int n_threads)
{
    orc_inst I;
    int rc = inst_prepare(P, lst, nu, &I);
    if (rc) return rc;
    const int nfd = P->n_feed, nax = P->n_ax, na = P->n_ant;
    const int64_t K = I.n_live;
    const int64_t N = (int64_t)nfd * na;
    int64_t npairs = n_pairs < 0 ? (int64_t)na * na : n_pairs;
    const double kappa = nu / ORC_C_LIGHT; /* turns per metre of delay path */
    int bad = 0;
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads) reduction(| : bad)
    for (int64_t q = 0; q < npairs; ++q) {
        int a, b;
        if (n_pairs < 0) { a = (int)(q / na); b = (int)(q % na); }
        else { a = pa[q]; b = pb[q]; }
        if (a < 0 || a >= na || b < 0 || b >= na) { bad = 1; continue; }
        int ba = P->beam_kind >= 2 && P->beam_idx ? P->beam_idx[a] : 0;
        int bb = P->beam_kind >= 2 && P->beam_idx ? P->beam_idx[b] : 0;
        double bx = P->enu[3 * a] - P->enu[3 * b];
        double by = P->enu[3 * a + 1] - P->enu[3 * b + 1];
        double bz = P->enu[3 * a + 2] - P->enu[3 * b + 2];
        double acc[4][2];
        memset(acc, 0, sizeof(acc));
        for (int64_t s = 0; s < K; ++s) {
            const double *x = &I.enu[3 * s];
            double tau = (bx * x[0] + by * x[1]) + bz * x[2];   /* metres */
            double phase = -2.0 * ORC_PI * kappa * tau;
            double c = cos(phase), sn = sin(phase);
            for (int p = 0; p < nfd; ++p)
                for (int r = 0; r < nfd; ++r) {
                    double tr = 0.0, ti = 0.0;
                    for (int k = 0; k < nax; ++k) {
                        const double *u = &I.A[2 * ((((int64_t)ba * nfd + p) * nax + k) * K + s)];
                        const double *v = &I.A[2 * ((((int64_t)bb * nfd + r) * nax + k) * K + s)];
                        /* u * conj(v) */
                        tr += u[0] * v[0] + u[1] * v[1];
                        ti += u[1] * v[0] - u[0] * v[1];
                    }
                    double f = I.flux[s];
                    acc[p * nfd + r][0] += f * (tr * c - ti * sn);
                    acc[p * nfd + r][1] += f * (tr * sn + ti * c);
                }
        }
        for (int p = 0; p < nfd; ++p)
            for (int r = 0; r < nfd; ++r) {
                int64_t o;
                if (n_pairs < 0) o = ((int64_t)a * nfd + p) * N + (int64_t)b * nfd + r;
                else o = (q * nfd + p) * nfd + r;
                out[2 * o] = acc[p * nfd + r][0];
                out[2 * o + 1] = acc[p * nfd + r][1];
            }
    }
    inst_free(&I);
    return bad ? -2 : 0;
}

/* Outer-product form (Algorithm 2 steps iii-v): builds
 * Z[(a,p)][(s,k)] = sqrt(I_s) A_{beta(a)}^{pk}(s) exp(-2 pi i (nu/c) x_a . X_hrz,s)
 * (eq. "littlez") in FP64 and forms V = Z Z^dagger (eq. "zz") with a plain
 * triple loop.  A cross-check of the direct sum on small problems only.
 * out complex128 [N][N]. */
int orc_vis_outer(const orc_problem *P, double lst, double nu, double *out)
{
    orc_inst I;
    int rc = inst_prepare(P, lst, nu, &I);
    if (rc) return rc;
    const int nfd = P->n_feed, nax = P->n_ax, na = P->n_ant;
    const int64_t K = I.n_live, N = (int64_t)nfd * na, M = K * nax;
    const double kappa = nu / ORC_C_LIGHT;
    double *Z = malloc(sizeof(double) * 2 * (size_t)(N > 0 ? N : 1) * (M > 0 ? M : 1));
    for (int a = 0; a < na; ++a) {
        int ba = P->beam_kind >= 2 && P->beam_idx ? P->beam_idx[a] : 0;
        for (int64_t s = 0; s < K; ++s) {
            const double *x = &I.enu[3 * s];
            double tau = (P->enu[3 * a] * x[0] + P->enu[3 * a + 1] * x[1]) + P->enu[3 * a + 2] * x[2];
            double phase = -2.0 * ORC_PI * kappa * tau;
            double c = cos(phase), sn = sin(phase), w = sqrt(I.flux[s]);
            for (int p = 0; p < nfd; ++p)
                for (int k = 0; k < nax; ++k) {
                    const double *u = &I.A[2 * ((((int64_t)ba * nfd + p) * nax + k) * K + s)];
                    int64_t o = ((int64_t)a * nfd + p) * M + s * nax + k;
                    Z[2 * o] = w * (u[0] * c - u[1] * sn);
                    Z[2 * o + 1] = w * (u[0] * sn + u[1] * c);
                }
        }
    }
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            double sr = 0.0, si = 0.0;
            for (int64_t m = 0; m < M; ++m) {
                const double *u = &Z[2 * (i * M + m)], *v = &Z[2 * (j * M + m)];
                sr += u[0] * v[0] + u[1] * v[1];
                si += u[1] * v[0] - u[0] * v[1];
            }
            out[2 * (i * N + j)] = sr;
            out[2 * (i * N + j) + 1] = si;
        }
    free(Z);
    inst_free(&I);
    return 0;
}
