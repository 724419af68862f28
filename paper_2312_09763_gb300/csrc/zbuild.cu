// zbuild.cu -- Algorithm 2 steps (iii)-(iv) of arXiv:2312.09763 (Sec. 3.1):
// the antenna-based phase tau = -2 pi i nu D X_hrz / c and the per-antenna
// matrix Z[(a,p),(s,k)] = sqrt(I_s) A^{pk}_{beta(a)}(s) exp(tau_as) of
// eq. "littlez" (Sec. 2.2), written as the real matrix U with interleaved
// rows 2(a n_feed + p) = Re Z, 2(a n_feed + p) + 1 = Im Z and columns
// s n_ax + k, so that V = Z Z^dagger becomes the real product U U^T.
//
// The phase argument (nu/c) x_a . s_hat is formed in FP64 and reduced
// exactly modulo one turn into 64-bit fixed point (bit operations on the
// FP64 significand); only the reduced fraction is rounded to FP32 for
// sincospi.  For the channels of one time that are equally spaced in nu,
// (x_a . s_hat) kappa_0 and (x_a . s_hat) dkappa are formed in FP64 once per
// (antenna, source) and the channel phases are stepped by exact 64-bit
// integer addition of their fractions.
#include <cuda_fp16.h>
#include "common.cuh"

namespace mv {
namespace {

// frac(p) * 2^64 modulo 2^64 for an FP64 value p: exact for |p| >= 2^-11,
// truncated below 2^-64 turns otherwise.
__device__ __forceinline__ unsigned long long frac64(double p) {
    const long long b = __double_as_longlong(p);
    const int ex = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1075 - ex;  // |p| = mant * 2^-sh
    unsigned long long f;
    if (ex == 0 || sh <= 0 || sh >= 117) f = 0ull;
    else if (sh <= 64) f = mant << (64 - sh);
    else f = mant >> (sh - 64);
    return b < 0 ? (0ull - f) : f;
}

// Fixed-point turns in [-1/2, 1/2) as FP32 (top 32 bits, two's complement).
__device__ __forceinline__ float turns(unsigned long long f) {
    return (float)(int)(f >> 32) * 2.3283064365386962890625e-10f;  // 2^-32
}

// Store one real entry of U: FP32 (PREC 0), or split into hi + lo halves,
// BF16 (PREC 1) or FP16 after the instance's power-of-two scale (PREC 2).
template <int PREC>
__device__ __forceinline__ void put(void* u, void* ulo, long long o, float v, float scale) {
    if (PREC == 0) {
        static_cast<float*>(u)[o] = v;
    } else if (PREC == 1) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        static_cast<__nv_bfloat16*>(u)[o] = hi;
        static_cast<__nv_bfloat16*>(ulo)[o] = lo;
    } else {
        const float x = v * scale;
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        static_cast<__half*>(u)[o] = hi;
        static_cast<__half*>(ulo)[o] = lo;
    }
}

template <int PREC>
__global__ void __launch_bounds__(128)
k_zbuild(Model m, const Inst* __restrict__ inst, const Chan* __restrict__ chan,
         const ZGroup* __restrict__ groups, int g_first, LiveTables lt, const float2* __restrict__ wa,
         long long wa_pitch, const float* __restrict__ amax, void* u, void* ulo, int rows, long long k_pitch,
         int ant_per_block) {
    const ZGroup g = groups[g_first + blockIdx.z];
    const int slot0 = g.slot0;
    const int t = inst[g.inst0].t;
    const int nl = lt.n_live[t];
    const long long kpad = ((long long)nl * m.n_ax + kKPad - 1) / kKPad * kKPad;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if ((long long)s * m.n_ax >= kpad) return;
    const int a_begin = blockIdx.y * ant_per_block;
    const int a_end = min(m.n_ant, a_begin + ant_per_block);
    const long long slot_stride = (long long)rows * k_pitch;
    const int ncomp = m.n_beam * m.n_feed * m.n_ax;
    if (s >= nl) {  // zero padding of the source axis up to the k granularity
        for (int j = 0; j < g.n; ++j) {
            const long long base = (long long)(slot0 + j) * slot_stride;
            for (int a = a_begin; a < a_end; ++a)
                for (int p = 0; p < m.n_feed; ++p)
                    for (int k = 0; k < m.n_ax; ++k) {
                        const long long r = 2ll * (a * m.n_feed + p);
                        const long long col = (long long)s * m.n_ax + k;
                        put<PREC>(u, ulo, base + r * k_pitch + col, 0.f, 1.f);
                        put<PREC>(u, ulo, base + (r + 1) * k_pitch + col, 0.f, 1.f);
                    }
        }
        return;
    }
    const long long lo = (long long)t * lt.pitch + s;
    const double se = lt.e[lo], sn = lt.n[lo], su = lt.u[lo];
    for (int a = a_begin; a < a_end; ++a) {
        // path length x_a . s_hat in metres (FP64)
        const double d = fma(m.ant_e[a], se, fma(m.ant_n[a], sn, m.ant_u[a] * su));
        const int beta = m.beam_idx[a];
        unsigned long long F = 0ull, FQ = 0ull;
        if (g.uniform) {
            F = frac64(d * g.kappa0);
            FQ = frac64(d * g.dkappa);
        }
        for (int j = 0; j < g.n; ++j) {
            if (!g.uniform) F = frac64(d * chan[inst[g.inst0 + j].c].kappa);
            float sv, cv;
            sincospif(2.f * turns(F), &sv, &cv);  // exp(-2 pi i p) = cv - i sv
            const int slot = slot0 + j;
            const long long base = (long long)slot * slot_stride;
            const float scale = PREC == 2 ? ldexpf(1.f, fp16_scale_exp(amax[slot])) : 1.f;
            const float2* w = wa + ((long long)slot * ncomp + (long long)beta * m.n_feed * m.n_ax) * wa_pitch + s;
            for (int p = 0; p < m.n_feed; ++p)
                for (int k = 0; k < m.n_ax; ++k) {
                    const float2 A = w[(long long)(p * m.n_ax + k) * wa_pitch];
                    const float re = fmaf(A.x, cv, A.y * sv);
                    const float im = fmaf(A.y, cv, -A.x * sv);
                    const long long r = 2ll * (a * m.n_feed + p);
                    const long long col = (long long)s * m.n_ax + k;
                    put<PREC>(u, ulo, base + r * k_pitch + col, re, scale);
                    put<PREC>(u, ulo, base + (r + 1) * k_pitch + col, im, scale);
                }
            F += FQ;
        }
    }
}

}  // namespace

cudaError_t launch_zbuild(const Model& m, const Inst* d_inst, const Chan* d_chan, const ZGroup* d_groups,
                          int g_first, int n_groups, LiveTables lt, const float2* d_wa, long long wa_pitch,
                          const float* d_amax, void* d_u, void* d_u_lo, int prec, int rows, long long k_pitch,
                          cudaStream_t st, long long* launches) {
    const int apb = 32;
    dim3 grid((unsigned)((lt.pitch + 127) / 128), (m.n_ant + apb - 1) / apb, n_groups);
    if (prec == 0)
        k_zbuild<0><<<grid, 128, 0, st>>>(m, d_inst, d_chan, d_groups, g_first, lt, d_wa, wa_pitch, d_amax, d_u,
                                          nullptr, rows, k_pitch, apb);
    else if (prec == 1)
        k_zbuild<1><<<grid, 128, 0, st>>>(m, d_inst, d_chan, d_groups, g_first, lt, d_wa, wa_pitch, d_amax, d_u,
                                          d_u_lo, rows, k_pitch, apb);
    else
        k_zbuild<2><<<grid, 128, 0, st>>>(m, d_inst, d_chan, d_groups, g_first, lt, d_wa, wa_pitch, d_amax, d_u,
                                          d_u_lo, rows, k_pitch, apb);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
