// perturb.cu -- the "fast" coordinate scheme of Algorithm 1 (Sec. 2.3 of
// arXiv:2312.09763), steps (ii) and (iv)-(vi), on the host in FP64.
//
// The rigid rotation of eq. "rotation" misses the time-dependent astrometric
// corrections (precession, nutation, aberration, ...).  Algorithm 1 moves
// every source to fictitious equatorial coordinates such that the rigid
// rotation at a reference time t_ref puts it exactly where an accurate
// transform puts it:
//   (i)   apparent LST at t_ref                       -- the caller's (astropy)
//   (ii)  R'(t_ref) = R(t_ref)^-1 = R(t_ref)^T (R is orthonormal)
//   (iii) apparent (alt, az) of each source at t_ref  -- the caller's (astropy)
//   (iv)  X_hrz = (cos alt sin az, cos alt cos az, sin alt) in East-North-Up,
//         az measured from North through East (the library's convention)
//   (v)   X_eq' = R'(t_ref) X_hrz
//   (vi)  RA' = atan2(y, x) in [0, 2 pi), Dec' = atan2(z, sqrt(x^2 + y^2)),
//         the inverse of eq. "xeq".
// Simulating at LST_ref with (RA', Dec') then reproduces X_hrz to rounding;
// the correction degrades away from t_ref, so long runs are cut into chunks
// of time, each with its own reference time and perturbed catalogue.
#include <cmath>
#include <cstdio>

#include "matvis.h"
#include "common.cuh"

extern "C" mv_status mv_perturb_sky(int64_t n_src, const double* alt_rad, const double* az_rad, double lst_ref_rad,
                                    double latitude_rad, double* ra_out, double* dec_out) {
    mv::set_last_error("");
    if (n_src < 1) {
        mv::set_last_error("mv_perturb_sky: n_src must be >= 1");
        return MV_ERR_ARG;
    }
    if (!alt_rad || !az_rad || !ra_out || !dec_out) {
        mv::set_last_error("mv_perturb_sky: NULL pointer argument");
        return MV_ERR_ARG;
    }
    if (!std::isfinite(lst_ref_rad) || !std::isfinite(latitude_rad) || std::fabs(latitude_rad) > 0.5 * mv::kPi) {
        mv::set_last_error("mv_perturb_sky: LST must be finite and |latitude| <= pi/2");
        return MV_ERR_ARG;
    }
    for (int64_t s = 0; s < n_src; ++s) {
        if (!std::isfinite(alt_rad[s]) || !std::isfinite(az_rad[s]) || std::fabs(alt_rad[s]) > 0.5 * mv::kPi) {
            char msg[128];
            snprintf(msg, sizeof(msg), "mv_perturb_sky: (alt, az)[%lld] not finite or |alt| > pi/2", (long long)s);
            mv::set_last_error(msg);
            return MV_ERR_ARG;
        }
    }
    // (ii) R(t_ref) of eq. "rotation" (H = -LST, rows East, North, Up); its
    // inverse is its transpose
    const double H = -lst_ref_rad;
    const double sH = std::sin(H), cH = std::cos(H), sl = std::sin(latitude_rad), cl = std::cos(latitude_rad);
    const double R[3][3] = {{sH, cH, 0.0}, {-sl * cH, sl * sH, cl}, {cl * cH, -cl * sH, sl}};
    const double two_pi = 2.0 * mv::kPi;
    for (int64_t s = 0; s < n_src; ++s) {
        // (iv) apparent direction in East-North-Up
        const double ca = std::cos(alt_rad[s]);
        const double h[3] = {ca * std::sin(az_rad[s]), ca * std::cos(az_rad[s]), std::sin(alt_rad[s])};
        // (v) X_eq' = R^T X_hrz
        double x[3];
        for (int i = 0; i < 3; ++i) x[i] = R[0][i] * h[0] + R[1][i] * h[1] + R[2][i] * h[2];
        // (vi) inverse of eq. "xeq"
        double ra = std::atan2(x[1], x[0]);
        if (ra < 0.0) ra += two_pi;
        if (ra >= two_pi) ra -= two_pi;
        ra_out[s] = ra;
        dec_out[s] = std::atan2(x[2], std::hypot(x[0], x[1]));
    }
    return MV_OK;
}
