// zcore.cuh -- the per-element core of the Z build (Algorithm 2 steps
// (iii)-(iv) of arXiv:2312.09763, eq. "littlez" / eq. "fullz"), shared by the
// stand-alone Z-build kernel (zbuild.cu) and the Z-build warps that run inside
// the tensor-core HERK (herk_tc.cu) for the next batch.
//
// The phase argument frac((nu/c) x_a . s_hat) is formed in 64-bit fixed
// point (turns x 2^64) with integer arithmetic: per (wavenumber, antenna)
// y = (nu/c) x_a is split into Y = rint(y 2^32) (AntPhase, from FP64), per
// (time, source) s_hat into S = rint(s_hat 2^31) and a residual eps; the sum
// of Y S (a 96-bit integer) is taken modulo 2^63 with 32 x 32 -> 64-bit
// multiply-adds, and the small term y . eps is added in FP32 (its magnitude
// is below |y| 2^-31, so its rounding error is below 1e-13 turns for the
// arrays here).  The phase is exact to about 2^-32 turns, with no FP64
// arithmetic per element.  For the channels of one time that are equally
// spaced in nu, the phases at kappa_0 and dkappa are formed once per
// (antenna, source) and the channel phases advance by exact 64-bit integer
// addition.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace mv {
namespace zcore {

// frac(kappa x_a . s_hat) x 2^64 for one antenna factor p and one source
// (S[c] = S_c + 2^31, eps[c]).  With S_c = S'_c - 2^31:
//   sum_c Y_c S_c = sum_c yl_c S'_c - sum_c yl_c 2^31 + 2^32 sum_c yh_c S'_c  (mod 2^63),
// which is (acc << 1) below read in 2^-64 turns; the y . eps term is added
// after rounding to 2^-32 turns.
__device__ __forceinline__ unsigned long long phase64(const AntPhase& p, const unsigned* S, const float* eps) {
    unsigned long long acc = ((unsigned long long)p.negk_hi << 32) | p.negk_lo;
    acc += (unsigned long long)p.yl[0] * S[0];
    acc += (unsigned long long)p.yl[1] * S[1];
    acc += (unsigned long long)p.yl[2] * S[2];
    const unsigned h = (unsigned)p.yh[0] * S[0] + (unsigned)p.yh[1] * S[1] + (unsigned)p.yh[2] * S[2];
    acc += (unsigned long long)h << 32;
    const float corr = fmaf(p.yf[0], eps[0], fmaf(p.yf[1], eps[1], p.yf[2] * eps[2]));
    const int cf = __float2int_rn(corr * 4294967296.0f);  // 2^32
    return (acc << 1) + ((unsigned long long)(long long)cf << 32);
}

__device__ __forceinline__ AntPhase load_phase(const AntPhase* __restrict__ t) {
    const uint4* q = reinterpret_cast<const uint4*>(t);
    const uint4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    AntPhase p;
    p.yl[0] = a.x; p.yl[1] = a.y; p.yl[2] = a.z;
    p.yh[0] = (int)a.w; p.yh[1] = (int)b.x; p.yh[2] = (int)b.y;
    p.yf[0] = __uint_as_float(b.z); p.yf[1] = __uint_as_float(b.w); p.yf[2] = __uint_as_float(c.x);
    p.negk_lo = c.y; p.negk_hi = c.z; p.pad = 0;
    return p;
}

// cos(2 pi r), sin(2 pi r) for the fixed-point turn F (r = frac(F / 2^64)):
// the nearest quarter turn q comes from the top bits, the remainder
// x in [-1/8, 1/8) turns goes through polynomials fitted to sin(2 pi x) / x and
// cos(2 pi x) in x^2 (least squares on Chebyshev nodes, |error| < 2e-9 before
// FP32 rounding), and the result is rotated by q quarter turns.
__device__ __forceinline__ void cos_sin_turns(unsigned long long F, float& c, float& s) {
    const unsigned X = (unsigned)(F >> 32);
    const unsigned q = (X + 0x20000000u) >> 30;
    const int t = (int)(X - (q << 30));
    const float x = (float)t * 2.3283064365386962890625e-10f;  // 2^-32
    const float x2 = x * x;
    const float sp = fmaf(fmaf(fmaf(-75.24006652832031f, x2, 81.58812713623047f), x2, -41.34162902832031f), x2,
                          6.283185005187988f) * x;
    const float cp = fmaf(fmaf(fmaf(fmaf(59.22040557861328f, x2, -85.44285583496094f), x2, 64.93931579589844f), x2,
                               -19.739208221435547f), x2, 1.0f);
    const bool swap = (q & 1u) != 0u;
    const float a = swap ? sp : cp, b = swap ? cp : sp;
    c = __int_as_float(__float_as_int(a) ^ (int)((((q + 1u) & 2u)) << 30));
    s = __int_as_float(__float_as_int(b) ^ (int)(((q & 2u)) << 30));
}

// Store 2 n_ax consecutive entries of one row of U (two sources): FP32
// (PREC 0), or the hi and lo FP16 halves of values already scaled (PREC 2) in
// the two planes.
template <int PREC, int NAX>
__device__ __forceinline__ void put_row(void* pu, void* pl, const float* v) {
    static_assert(PREC == 0 || PREC == 2, "FP32 or FP16 hi + lo");
    if constexpr (PREC == 0) {
        float* p = static_cast<float*>(pu);
        if constexpr (NAX == 1) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
        else *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        uint32_t hi[NAX], lo[NAX];
#pragma unroll
        for (int i = 0; i < NAX; ++i) {
            const float x0 = v[2 * i], x1 = v[2 * i + 1];
            const __half2 h = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(h);
            const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
            hi[i] = *reinterpret_cast<const uint32_t*>(&h);
            lo[i] = *reinterpret_cast<const uint32_t*>(&l);
        }
        if constexpr (NAX == 1) {
            *static_cast<uint32_t*>(pu) = hi[0];
            *static_cast<uint32_t*>(pl) = lo[0];
        } else {
            *static_cast<uint2*>(pu) = make_uint2(hi[0], hi[1]);
            *static_cast<uint2*>(pl) = make_uint2(lo[0], lo[1]);
        }
    }
}

// Channels between exact phase evaluations when the channels of a group are
// equally spaced: in between, cos(2 pi F) + i sin(2 pi F) advances by one
// complex product with e^{2 pi i dF} per channel (seven FP32 steps at most,
// each adding about 2^-23 relative error); the WA values of kPrefetch
// channels are loaded together.
constexpr int kAnchor = 8, kPrefetch = 4;

// Element type of the U planes.
template <int PREC> struct Plane { using T = uint16_t; };
template <> struct Plane<0> { using T = float; };

// One work item (bx, by, group g) of nthr threads: thread tid builds the two
// adjacent sources 2 (bx nthr + tid) and +1 (columns 2 n_ax wide) for antennas
// [by ant_per_block, +ant_per_block) and every instance of the group.
// Sources past the live count (up to the k padding) are written as zeros
// (their WA entries are zero).  scale[0]: the FP16 scale of the group (one
// power of two for all its instances), folded into the cos/sin factors.
template <int PREC, int NAX, int NFD>
__device__ __forceinline__ void zbuild_item(const Model& m, const Inst* __restrict__ inst, const ZGroup& g,
                                            const LiveTables& lt, const float2* __restrict__ wa,
                                            long long wa_pitch, const float* __restrict__ scale, void* u, void* ulo,
                                            int rows, long long k_pitch, int ant_per_block,
                                            const AntPhase* __restrict__ tab, int bx, int by, int nthr, int tid) {
    using T = typename Plane<PREC>::T;
    const int t = inst[g.inst0].t;
    const int nl = lt.n_live[t];
    const long long kpad = ((long long)nl * NAX + kKPad - 1) / kKPad * kKPad;
    const int s0 = 2 * (bx * nthr + tid);
    if ((long long)s0 * NAX >= kpad) return;
    const int a_begin = by * ant_per_block;
    const int a_end = min(m.n_ant, a_begin + ant_per_block);
    const long long slot_stride = (long long)rows * k_pitch;
    const long long wa_slot = (long long)m.n_beam * NFD * NAX * wa_pitch;
    const bool live0 = s0 < nl, live1 = s0 + 1 < nl;
    // the two sources' direction in fixed point (zeros past the live count)
    unsigned S0[3] = {0u, 0u, 0u}, S1[3] = {0u, 0u, 0u};
    float E0[3] = {0.f, 0.f, 0.f}, E1[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long o3 = ((long long)t * 3 + c) * lt.pitch + s0;
        if (live0) {
            const uint2 q = *reinterpret_cast<const uint2*>(lt.sfix + o3);
            const float2 r = *reinterpret_cast<const float2*>(lt.seps + o3);
            S0[c] = q.x; E0[c] = r.x;
            if (live1) { S1[c] = q.y; E1[c] = r.y; }
        }
    }
    const long long col = (long long)s0 * NAX;
    T* const ub = static_cast<T*>(u) + g.slot0 * slot_stride + col;
    T* const lb = PREC != 0 ? static_cast<T*>(ulo) + g.slot0 * slot_stride + col : nullptr;
    const float2* const wb = wa + g.slot0 * wa_slot + s0;
    const bool step = g.uniform && g.n > 1;
    const float sc = PREC == 2 ? scale[0] : 1.f;
    for (int a = a_begin; a < a_end; ++a) {
        const float2* w = wb + (long long)m.beam_idx[a] * (NFD * NAX) * wa_pitch;
        T* ur = ub + 2ll * a * NFD * k_pitch;
        T* lr = PREC != 0 ? lb + 2ll * a * NFD * k_pitch : nullptr;
        // WA of the two sources for the group's instance w + jrel: one 16-byte load
        // per component (s0 is even)
        constexpr int NC = NFD * NAX;
        auto load_wa = [&](int jrel, float4 (&A)[NC]) {
            const float2* wj = w + (long long)jrel * wa_slot;
#pragma unroll
            for (int c = 0; c < NC; ++c) A[c] = *reinterpret_cast<const float4*>(wj + (long long)c * wa_pitch);
        };
        // U rows 2(a NFD + p) + {0, 1} of the next instance of the group, at
        // phase (c, s) (times the FP16 scale)
        auto emit = [&](const float4 (&A)[NC], float c0, float sn0, float c1, float sn1) {
#pragma unroll
            for (int p = 0; p < NFD; ++p) {
                float re[2 * NAX], im[2 * NAX];
#pragma unroll
                for (int k = 0; k < NAX; ++k) {
                    const float4 a4 = A[p * NAX + k];
                    // Z = WA * exp(-2 pi i phase) = WA * (c - i s)
                    re[k] = fmaf(a4.x, c0, a4.y * sn0);
                    im[k] = fmaf(a4.y, c0, -a4.x * sn0);
                    re[NAX + k] = fmaf(a4.z, c1, a4.w * sn1);
                    im[NAX + k] = fmaf(a4.w, c1, -a4.z * sn1);
                }
                const long long r0 = 2ll * p * k_pitch;
                put_row<PREC, NAX>(ur + r0, PREC != 0 ? lr + r0 : nullptr, re);
                put_row<PREC, NAX>(ur + r0 + k_pitch, PREC != 0 ? lr + r0 + k_pitch : nullptr, im);
            }
            ur += slot_stride;
            if (PREC != 0) lr += slot_stride;
        };
        if (step) {
            // equally spaced channels: exact fixed-point phase every kAnchor
            // channels, complex recurrence in between
            const AntPhase p0 = load_phase(tab + a), pd = load_phase(tab + m.n_ant + a);
            unsigned long long F0 = phase64(p0, S0, E0), F1 = phase64(p0, S1, E1);
            const unsigned long long Q0 = phase64(pd, S0, E0), Q1 = phase64(pd, S1, E1);
            float rc0, rs0, rc1, rs1;
            cos_sin_turns(Q0, rc0, rs0);
            cos_sin_turns(Q1, rc1, rs1);
            for (int j0 = 0; j0 < g.n; j0 += kAnchor) {
                float c0, sn0, c1, sn1;
                cos_sin_turns(F0, c0, sn0);
                cos_sin_turns(F1, c1, sn1);
                c0 *= sc;
                sn0 *= sc;
                c1 *= sc;
                sn1 *= sc;
                F0 += Q0 * kAnchor;
                F1 += Q1 * kAnchor;
#pragma unroll
                for (int jb = 0; jb < kAnchor; jb += kPrefetch) {
                    // one-component beams: the WA loads of kPrefetch channels go out together
                    constexpr int PF = NC == 1 ? kPrefetch : 1;
                    float4 Apf[PF][NC];
                    if constexpr (PF > 1) {
#pragma unroll
                        for (int jj = 0; jj < PF; ++jj)
                            if (j0 + jb + jj < g.n) load_wa(jj, Apf[jj]);
                    }
#pragma unroll
                    for (int jj = 0; jj < kPrefetch; ++jj) {
                        if (j0 + jb + jj < g.n) {
                            if constexpr (PF > 1) {
                                emit(Apf[jj], c0, sn0, c1, sn1);
                            } else {
                                load_wa(jj, Apf[0]);
                                emit(Apf[0], c0, sn0, c1, sn1);
                            }
                        }
                        if (jb + jj + 1 < kAnchor) {  // (c + i s) e^{2 pi i dF}
                            const float nc0 = fmaf(c0, rc0, -sn0 * rs0), nc1 = fmaf(c1, rc1, -sn1 * rs1);
                            sn0 = fmaf(sn0, rc0, c0 * rs0);
                            sn1 = fmaf(sn1, rc1, c1 * rs1);
                            c0 = nc0;
                            c1 = nc1;
                        }
                    }
                    w += kPrefetch * wa_slot;
                }
            }
        } else {
            for (int j = 0; j < g.n; ++j) {
                const AntPhase pj = load_phase(tab + (long long)(g.uniform ? 0 : j) * m.n_ant + a);
                float4 A[NC];
                load_wa(0, A);
                float c0, sn0, c1, sn1;
                cos_sin_turns(phase64(pj, S0, E0), c0, sn0);
                cos_sin_turns(phase64(pj, S1, E1), c1, sn1);
                emit(A, c0 * sc, sn0 * sc, c1 * sc, sn1 * sc);
                w += wa_slot;
            }
        }
    }
}

// Z build of one batch by the warps of another kernel: work items of 64
// sources (one warp) x ant_per_block antennas x one group, taken in order
// (sources fastest, then antennas, then groups), item i by warp i mod n_warps.
// sw: 16 floats of this warp's shared memory for the group's FP16 scales.
template <int PREC, int NAX, int NFD>
__device__ __forceinline__ void zjob_warp(const ZJob& z, int warp_id, int n_warps, float* sw) {
    const int lane = threadIdx.x & 31;
    constexpr int apb = 32;
    const int nx = (int)((z.lt.pitch / 2 + 31) / 32), ny = (z.m.n_ant + apb - 1) / apb;
    const long long n_items = (long long)nx * ny * z.n_groups;
    for (long long item = warp_id; item < n_items; item += n_warps) {
        const int bx = (int)(item % nx);
        const long long rest = item / nx;
        const int by = (int)(rest % ny), bz = (int)(rest / ny);
        const ZGroup g = z.groups[z.g_first + bz];
        __syncwarp();
        if (PREC == 2 && lane < g.n) sw[lane] = ldexpf(1.f, fp16_scale_exp(z.amax[g.slot0 + lane]));
        __syncwarp();
        zbuild_item<PREC, NAX, NFD>(z.m, z.inst, g, z.lt, z.wa, z.wa_pitch, sw, z.u, z.ulo, z.rows, z.k_pitch, apb,
                                    z.aph + (long long)bz * z.n_phase * z.m.n_ant, bx, by, 32, lane);
    }
}

}  // namespace zcore
}  // namespace mv
