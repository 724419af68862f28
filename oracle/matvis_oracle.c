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
 * the case that leads to eq. "littlez").  With Stokes Q, U, V given, the
 * source term I_s sum_k A^{pk} conj(A^{qk}) becomes the full
 * sum_{k,k'} A^{pk} C_{kk'} conj(A^{qk'}) with the coherency of Sec. 2.1,
 * C = [[I + Q, U + iV], [U - iV, I - Q]] in the beam's (theta, phi) component
 * basis (eq. "matvistensorprod"), all four Stokes scaled by (nu/nu_ref)^alpha.  Source directions follow eq. "xeq"
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
    /* polarised sky (needs n_ax = 2): [3][n_src] Stokes Q, U, V in Jy at
     * nu_ref, or NULL for an unpolarised sky */
    const double *stokes_quv;
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

/* Algorithm 1 (Sec. 2.3), steps (ii) and (iv)-(vi): perturbed equatorial
 * coordinates from the apparent altitude and azimuth of each source at a
 * reference LST (steps (i) and (iii) belong to the caller).
 *   (ii)  R' = inverse of eq. "rotation" at (lst_ref, lat); R is orthonormal,
 *         so R' is its transpose, read here by swapping the indices of R;
 *   (iv)  X_hrz = (cos alt sin az, cos alt cos az, sin alt) in East-North-Up;
 *   (v)   X_eq' = R' X_hrz;
 *   (vi)  the inverse of eq. "xeq": Dec' from the z component, RA' from x, y.
 * Writes ra[n], dec[n] in radians, RA' in [0, 2 pi). */
void orc_perturb_sky(int64_t n, const double *alt, const double *az, double lst_ref, double lat,
                     double *ra, double *dec)
{
    double R[9];
    orc_rotation(lst_ref, lat, R);
    for (int64_t s = 0; s < n; ++s) {
        double h[3], x[3];
        h[0] = cos(alt[s]) * sin(az[s]);
        h[1] = cos(alt[s]) * cos(az[s]);
        h[2] = sin(alt[s]);
        for (int i = 0; i < 3; ++i) {
            /* (R^T h)_i = sum_j R_ji h_j */
            x[i] = 0.0;
            for (int j = 0; j < 3; ++j) x[i] += R[3 * j + i] * h[j];
        }
        double r = sqrt(x[0] * x[0] + x[1] * x[1]);
        double a = atan2(x[1], x[0]);
        if (a < 0.0) a += 2.0 * ORC_PI;
        ra[s] = a;
        dec[s] = atan2(x[2], r);
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
    double *quv;    /* [n_live][3] Q, U, V at nu, or NULL */
} orc_inst;

static void inst_free(orc_inst *I)
{
    free(I->enu); free(I->flux); free(I->A); free(I->idx); free(I->quv);
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
    if (P->stokes_quv) I->quv = malloc(sizeof(double) * 3 * mm);
    double *az = malloc(sizeof(double) * mm), *za = malloc(sizeof(double) * mm);
    int64_t j = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (!(enu[3 * s + 2] > 0.0)) continue;
        memcpy(&I->enu[3 * j], &enu[3 * s], 3 * sizeof(double));
        double alpha = P->spec_idx ? P->spec_idx[s] : 0.0;
        double g = pow(nu / P->nu_ref, alpha);
        I->flux[j] = P->flux_ref[s] * g;
        if (I->quv)
            for (int c = 0; c < 3; ++c) I->quv[3 * j + c] = P->stokes_quv[(int64_t)c * n + s] * g;
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
 * Returns 0, -1 (frequency outside the beam grid), -2 (bad index) or -3 (a
 * polarised sky with a single-axis beam). */
int orc_vis(const orc_problem *P, double lst, double nu, int64_t n_pairs,
            const int32_t *pa, const int32_t *pb, double *out, int n_threads)
{
    if (P->stokes_quv && P->n_ax != 2) return -3;
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
                    double tr = 0.0, ti = 0.0, f = I.flux[s];
                    if (I.quv) {
                        /* sum_{k,k'} u_k C_kk' conj(v_k'), C from (I, Q, U, V) */
                        const double *q3 = &I.quv[3 * s];
                        double Cr[2][2] = {{f + q3[0], q3[1]}, {q3[1], f - q3[0]}};
                        double Ci[2][2] = {{0.0, q3[2]}, {-q3[2], 0.0}};
                        for (int k = 0; k < 2; ++k)
                            for (int k2 = 0; k2 < 2; ++k2) {
                                const double *u = &I.A[2 * ((((int64_t)ba * nfd + p) * nax + k) * K + s)];
                                const double *v = &I.A[2 * ((((int64_t)bb * nfd + r) * nax + k2) * K + s)];
                                /* w = u * C_kk' */
                                double wr = u[0] * Cr[k][k2] - u[1] * Ci[k][k2];
                                double wi = u[0] * Ci[k][k2] + u[1] * Cr[k][k2];
                                tr += wr * v[0] + wi * v[1];
                                ti += wi * v[0] - wr * v[1];
                            }
                        f = 1.0;
                    } else {
                        for (int k = 0; k < nax; ++k) {
                            const double *u = &I.A[2 * ((((int64_t)ba * nfd + p) * nax + k) * K + s)];
                            const double *v = &I.A[2 * ((((int64_t)bb * nfd + r) * nax + k) * K + s)];
                            /* u * conj(v) */
                            tr += u[0] * v[0] + u[1] * v[1];
                            ti += u[1] * v[0] - u[0] * v[1];
                        }
                    }
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

/* A square root M of the coherency, M M^dagger = C (Sec. 2.2, "second
 * trick"): the lower-triangular Cholesky factor
 *   M = [[m00, 0], [m10, m11]],  m00 = sqrt(I + Q),  m10 = (U - iV) / m00,
 *   m11 = sqrt(I - Q - |m10|^2),
 * with m10 = 0 and m11 = sqrt(I - Q) when I + Q = 0 (then U = V = 0 for a
 * physical source).  Writes m00, m10 (re, im), m11. */
void orc_coherency_sqrt(double I, double Q, double U, double V, double *m)
{
    double a = I + Q;
    m[0] = a > 0.0 ? sqrt(a) : 0.0;
    if (m[0] > 0.0) {
        m[1] = U / m[0];
        m[2] = -V / m[0];
    } else {
        m[1] = 0.0;
        m[2] = 0.0;
    }
    double d = I - Q - (m[1] * m[1] + m[2] * m[2]);
    m[3] = d > 0.0 ? sqrt(d) : 0.0;
}

/* Outer-product form (Algorithm 2 steps iii-v): builds
 * Z[(a,p)][(s,k)] = sqrt(I_s) A_{beta(a)}^{pk}(s) exp(-2 pi i (nu/c) x_a . X_hrz,s)
 * (eq. "littlez"), or for a polarised sky
 * Z[(a,p)][(s,k'')] = sum_k A^{pk}(s) F_as M_{kk''}(s) (eq. "fullz") with M from
 * orc_coherency_sqrt, in FP64 and forms V = Z Z^dagger (eq. "zz") with a
 * plain triple loop.  A cross-check of the direct sum on small problems
 * only.  out complex128 [N][N]. */
int orc_vis_outer(const orc_problem *P, double lst, double nu, double *out)
{
    if (P->stokes_quv && P->n_ax != 2) return -3;
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
            double m[4];
            if (I.quv) orc_coherency_sqrt(I.flux[s], I.quv[3 * s], I.quv[3 * s + 1], I.quv[3 * s + 2], m);
            for (int p = 0; p < nfd; ++p) {
                /* A^{pk} F for both axes */
                double af[2][2];
                for (int k = 0; k < nax; ++k) {
                    const double *u = &I.A[2 * ((((int64_t)ba * nfd + p) * nax + k) * K + s)];
                    af[k][0] = u[0] * c - u[1] * sn;
                    af[k][1] = u[0] * sn + u[1] * c;
                }
                for (int k = 0; k < nax; ++k) {
                    int64_t o = ((int64_t)a * nfd + p) * M + s * nax + k;
                    if (!I.quv) {
                        Z[2 * o] = w * af[k][0];
                        Z[2 * o + 1] = w * af[k][1];
                    } else if (k == 0) {  /* A0 M00 + A1 M10 */
                        Z[2 * o] = af[0][0] * m[0] + (af[1][0] * m[1] - af[1][1] * m[2]);
                        Z[2 * o + 1] = af[0][1] * m[0] + (af[1][0] * m[2] + af[1][1] * m[1]);
                    } else {              /* A1 M11 */
                        Z[2 * o] = af[1][0] * m[3];
                        Z[2 * o + 1] = af[1][1] * m[3];
                    }
                }
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
