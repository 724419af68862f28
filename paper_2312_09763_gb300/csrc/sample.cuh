// sample.cuh -- the training samples of the learned beam: where a sample
// lies (beam, az, za, nu) and its target, the gridded beam's own Keys-cubic
// interpolation (Sec. 2.4 of arXiv:2312.09763).  Used by the sampler kernel
// of mlp.cu, which draws the next training step's samples on the SMs the
// fused training pass leaves free; every sample comes from its own counters,
// so a batch is the same whichever SMs draw it.
#pragma once
#include "common.cuh"

namespace mv {

// splitmix64 (Steele, Lea and Flood 2014): a counter-based stream of 64-bit
// values; uniform floats in [0, 1) take its top 24 bits (FP32 only: the
// sampler does no FP64 arithmetic, which this GPU runs at a small fraction of
// its FP32 rate).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ __forceinline__ float uniform01f(unsigned long long seed, unsigned long long ctr) {
    return (float)(unsigned)(splitmix64(seed ^ splitmix64(ctr)) >> 40) * (1.0f / 16777216.0f);
}

// Where training samples may lie in frequency: the grid's fractional frequency
// index u = (nu - nu0) / dnu in [u_lo, u_lo + u_span) (inside the cubic
// stencil's margin), nu = nu0 + u dnu.
struct SampleRange {
    float u_lo, u_span, nu0, dnu;
};

struct Sample {
    int a;          // beam
    float az, za;   // radians
    float u, nu;    // fractional frequency index of the grid, Hz
};

// Sample i of the M of training step `step`: beams stratified over the batch
// (rows [b M / n_beam, (b + 1) M / n_beam) belong to beam b: each beam equally
// often, its rows together), az in [0, 2 pi), za in [0, pi/2) and u uniform.
__device__ __forceinline__ Sample draw_sample(unsigned long long seed, unsigned long long step, int M, int i,
                                              int n_beam, const SampleRange& rg) {
    const unsigned long long base = (step * (unsigned long long)M + i) * 4ull;
    Sample d;
    d.a = min(n_beam - 1, (int)(((long long)i * n_beam) / M));
    d.az = uniform01f(seed, base + 1) * 6.2831853f;
    d.za = uniform01f(seed, base + 2) * 1.5707963f;
    d.u = rg.u_lo + uniform01f(seed, base + 3) * rg.u_span;
    d.nu = rg.nu0 + d.u * rg.dnu;
    return d;
}

__device__ __forceinline__ float keys_w(float x) {
    const float t = fabsf(x);
    if (t <= 1.f) return (1.5f * t - 2.5f) * t * t + 1.f;
    if (t < 2.f) return ((-0.5f * t + 2.5f) * t - 4.f) * t + 2.f;
    return 0.f;
}

// Keys-cubic interpolation in (za, az) of component `comp` of beam `b` of the
// raw grid at frequency node f (pole and az wrap as in the beam step of the
// simulator).
__device__ __forceinline__ float2 grid_value_node(const Model& m, const float2* __restrict__ grid, int b, int comp,
                                                  float az, float za, int f) {
    const long long plane = (long long)m.n_za * m.n_az;
    const float2* G = grid + (((long long)b * m.n_feed * m.n_ax + comp) * m.n_nu + f) * plane;
    const float uz = za / m.dza, ua = az / m.daz;
    const float fz = floorf(uz), fa = floorf(ua);
    const float tz = uz - fz, ta = ua - fa;
    const int z0 = (int)fz - 1, a0 = (int)fa - 1;
    const float wz[4] = {keys_w(tz + 1.f), keys_w(tz), keys_w(1.f - tz), keys_w(2.f - tz)};
    const float wa[4] = {keys_w(ta + 1.f), keys_w(ta), keys_w(1.f - ta), keys_w(2.f - ta)};
    const float pole_sign = m.n_ax == 2 ? -1.f : 1.f;
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int row = z0 + r, sh = 0;
        float sg = 1.f;
        if (row < 0) { row = -row; sh = m.n_az / 2; sg = pole_sign; }
        if (row > m.n_za - 1) row = m.n_za - 1;
        // the row's four columns from c0 on, az wrapped into [0, n_az)
        int c0 = a0 + sh;
        if (c0 >= m.n_az) c0 -= m.n_az;
        if (c0 < 0) c0 += m.n_az;
        const float2* R = G + (long long)row * m.n_az;  // 16-byte aligned (n_az even)
        float2 v[4];
        if (c0 + 3 < m.n_az) {
            // unwrapped: two or three vector loads instead of four
            if ((c0 & 1) == 0) {
                const float4 p = *reinterpret_cast<const float4*>(R + c0);
                const float4 q = *reinterpret_cast<const float4*>(R + c0 + 2);
                v[0] = make_float2(p.x, p.y); v[1] = make_float2(p.z, p.w);
                v[2] = make_float2(q.x, q.y); v[3] = make_float2(q.z, q.w);
            } else {
                const float4 p = *reinterpret_cast<const float4*>(R + c0 + 1);
                v[0] = R[c0];
                v[1] = make_float2(p.x, p.y); v[2] = make_float2(p.z, p.w);
                v[3] = R[c0 + 3];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int col = c0 + q;
                if (col >= m.n_az) col -= m.n_az;
                v[q] = R[col];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float w2 = wz[r] * wa[q] * sg;
            re = fmaf(w2, v[q].x, re);
            im = fmaf(w2, v[q].y, im);
        }
    }
    return make_float2(re, im);
}

// Work item q of drawing M samples (four consecutive lanes per (sample,
// component), one per frequency node of the cubic stencil, summed with
// shuffles; every lane of a sample draws the same values).  All 32 lanes of a
// warp must call it together, with q = base + lane for a base that is a
// multiple of 4 (items q >= 4 M ncomp only take part in the shuffles).
__device__ __forceinline__ void sample_item(const Model& m, const float2* __restrict__ grid, const SampleRange& rg,
                                            unsigned long long seed, unsigned long long step, int M, int n_out,
                                            long long q, int* __restrict__ ant, float* __restrict__ az,
                                            float* __restrict__ za, float* __restrict__ nu, float* __restrict__ T) {
    const int ncomp = m.n_feed * m.n_ax;
    const int jt = (int)(q & 3);
    const long long qc = q >> 2;
    const bool valid = qc < (long long)M * ncomp;
    const int i = valid ? (int)(qc / ncomp) : 0, c = valid ? (int)(qc % ncomp) : 0;
    const Sample d = draw_sample(seed, step, M, i, m.n_beam, rg);
    float2 v = make_float2(0.f, 0.f);
    if (valid && 2 * c < n_out) {
        const float fu = floorf(d.u), tu = d.u - fu;
        const float w = keys_w(tu + 1.f - (float)jt);
        v = grid_value_node(m, grid, d.a, c, d.az, d.za, (int)fu - 1 + jt);
        v.x *= w;
        v.y *= w;
    }
    v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
    v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
    if (!valid || jt != 0) return;
    if (c == 0) {
        ant[i] = d.a;
        az[i] = d.az;
        za[i] = d.za;
        nu[i] = d.nu;
    }
    if (2 * c < n_out) {
        T[(long long)i * n_out + 2 * c] = v.x;
        T[(long long)i * n_out + 2 * c + 1] = v.y;
    }
}

}  // namespace mv
