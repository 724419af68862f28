// prep.cu -- Algorithm 2 steps (i) and (ii) of arXiv:2312.09763 (Sec. 3.1):
// rotation of the sources to East-North-Up with R(t) of eq. "rotation"
// (Sec. 2.3), the horizon cut with stable stream compaction, and the beam
// evaluation at the live sources (Sec. 2.4), fused with sqrt(I_s(nu)).
#include "common.cuh"

namespace mv {
namespace {

constexpr int kCullThreads = 256;

// One component of X_hrz = R X_eq, evaluated as (R0 x + R1 y) + R2 z with
// every product and sum rounded on its own (no FMA contraction), so the
// horizon decision Up > 0 is taken on a value fixed by that expression.
__device__ __forceinline__ double rot_row(const double* r, double x, double y, double z) {
    return __dadd_rn(__dadd_rn(__dmul_rn(r[0], x), __dmul_rn(r[1], y)), __dmul_rn(r[2], z));
}

__global__ void __launch_bounds__(kCullThreads)
k_cull_count(Model m, const double* __restrict__ R, int* __restrict__ counts, int bpt) {
    const int t = blockIdx.y;
    const long long s = (long long)blockIdx.x * kCullThreads + threadIdx.x;
    int live = 0;
    if (s < m.n_src) {
        const double* r = R + 9 * t;
        double up = rot_row(r + 6, m.xeq[s], m.xeq[m.n_src + s], m.xeq[2 * m.n_src + s]);
        live = up > 0.0;
    }
    int c = __syncthreads_count(live);
    if (threadIdx.x == 0) counts[(long long)t * bpt + blockIdx.x] = c;
}

// Exclusive scan of the per-block live counts of one time (one block per time).
__global__ void __launch_bounds__(1024)
k_cull_scan(const int* __restrict__ counts, int* __restrict__ offsets, int* __restrict__ n_live, int bpt) {
    __shared__ int warp_sums[32];
    const int t = blockIdx.x;
    const int per = (bpt + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    const int* c = counts + (long long)t * bpt;
    int local = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < bpt) local += c[b0 + i];
    // block exclusive scan of `local`
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int base = (warp > 0 ? warp_sums[warp - 1] : 0) + incl - local;
    int* o = offsets + (long long)t * bpt;
    for (int i = 0; i < per; ++i)
        if (b0 + i < bpt) { o[b0 + i] = base; base += c[b0 + i]; }
    if (threadIdx.x == blockDim.x - 1) n_live[t] = warp_sums[(blockDim.x >> 5) - 1];
}

__global__ void __launch_bounds__(kCullThreads)
k_cull_scatter(Model m, const double* __restrict__ R, const int* __restrict__ offsets, int bpt,
               LiveTables lt) {
    __shared__ int warp_base[kCullThreads / 32];
    const int t = blockIdx.y;
    const long long s = (long long)blockIdx.x * kCullThreads + threadIdx.x;
    double e = 0, n = 0, u = 0;
    int live = 0;
    if (s < m.n_src) {
        const double* r = R + 9 * t;
        const double x = m.xeq[s], y = m.xeq[m.n_src + s], z = m.xeq[2 * m.n_src + s];
        e = rot_row(r, x, y, z);
        n = rot_row(r + 3, x, y, z);
        u = rot_row(r + 6, x, y, z);
        live = u > 0.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned mask = __ballot_sync(0xffffffffu, live);
    if (lane == 0) warp_base[warp] = __popc(mask);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < kCullThreads / 32; ++w) { int c = warp_base[w]; warp_base[w] = acc; acc += c; }
    }
    __syncthreads();
    if (!live) return;
    const long long pos = (long long)offsets[(long long)t * bpt + blockIdx.x] + warp_base[warp] +
                          __popc(mask & ((1u << lane) - 1u));
    const long long o = (long long)t * lt.pitch + pos;
    lt.e[o] = e;
    lt.n[o] = n;
    lt.u[o] = u;
    lt.idx[o] = (int)s;
    if (lt.sfix) {
        const double comp[3] = {e, n, u};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double q = fmin(rint(comp[c] * 2147483648.0), 2147483647.0);  // 2^31
            const long long o3 = ((long long)t * 3 + c) * lt.pitch + pos;
            lt.sfix[o3] = (unsigned)((long long)q + 2147483648ll);
            lt.seps[o3] = (float)(comp[c] - q * 4.656612873077392578125e-10);  // 2^-31
        }
    }
    // az = atan2(E, N) in [0, 2 pi), za = atan2(|EN|, Up): well conditioned at the pole
    const float ef = (float)e, nf = (float)n, uf = (float)u;
    float az = atan2f(ef, nf);
    if (az < 0.f) az += 6.2831853071795864769f;
    const float za = atan2f(sqrtf(ef * ef + nf * nf), uf);
    lt.azza[o] = make_float2(az, za);
}

// Per-channel beam planes: P[c][b][p][k][za][az] = sum_m w_m(c) G[b][p][k][m0(c)+m][za][az]
// (the frequency axis of the gridded beam interpolated once per channel).
__global__ void k_beam_planes(Model m, const float2* __restrict__ grid, const Chan* __restrict__ chan,
                              float2* __restrict__ planes) {
    const long long plane = (long long)m.n_za * m.n_az;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int comp = blockIdx.y;  // (b, p, k) flattened
    const int c = blockIdx.z;
    const Chan ch = chan[c];
    const float2* g = grid + (long long)comp * m.n_nu * plane;
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 v = g[(long long)(ch.m0 + j) * plane + i];
        re = fmaf(ch.w[j], v.x, re);
        im = fmaf(ch.w[j], v.y, im);
    }
    const int n_comp = gridDim.y;
    planes[((long long)c * n_comp + comp) * plane + i] = make_float2(re, im);
}

// Keys (1981) cubic-convolution kernel, a = -1/2.
__device__ __forceinline__ float keys(float x) {
    const float t = fabsf(x);
    if (t <= 1.f) return (1.5f * t - 2.5f) * t * t + 1.f;
    if (t < 2.f) return ((-0.5f * t + 2.5f) * t - 4.f) * t + 2.f;
    return 0.f;
}

// WA[slot][b][p][k][s] = sqrt(I_s(nu)) * A^{pk}_b(az_s, za_s, nu) for the live
// sources of each instance (Algorithm 2 step ii, with the flux weight of step iv).
// Max of |value| over a warp, folded into amax (non-negative floats order
// like their bit patterns).
__device__ __forceinline__ void fold_amax(float v, float* amax) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(reinterpret_cast<int*>(amax), __float_as_int(v));
}

__device__ float wa_eval(const Model& m, const float2* __restrict__ planes, const Chan& ch, const Inst& in,
                         LiveTables lt, int s, float2* __restrict__ out, long long wa_pitch);

__global__ void __launch_bounds__(128)
k_wa(Model m, const float2* __restrict__ planes, const Chan* __restrict__ chan,
     const Inst* __restrict__ inst, int inst0, LiveTables lt, float2* __restrict__ wa, long long wa_pitch,
     float* __restrict__ amax) {
    const int slot = blockIdx.y;
    const Inst in = inst[inst0 + slot];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = lt.n_live[in.t];
    const int ncomp = m.n_beam * m.n_feed * m.n_ax;
    float mx = 0.f;
    float2* out = wa + (long long)slot * ncomp * wa_pitch + s;
    if (s < nl) {
        mx = wa_eval(m, planes, chan[in.c], in, lt, s, out, wa_pitch);
    } else if (s < wa_pitch) {  // zeros past the live count: the Z build reads whole source pairs
        for (int comp = 0; comp < ncomp; ++comp) out[(long long)comp * wa_pitch] = make_float2(0.f, 0.f);
    }
    fold_amax(mx, amax + slot);
}

// sqrt(I_s(nu)) A^{pk}_b(s) for every component of one live source; returns
// the largest magnitude written.
__device__ float wa_eval(const Model& m, const float2* __restrict__ planes, const Chan& ch, const Inst& in,
                         LiveTables lt, int s, float2* __restrict__ out, long long wa_pitch) {
    const long long o = (long long)in.t * lt.pitch + s;
    const int src = lt.idx[o];
    const float2 azza = lt.azza[o];
    const float spec = expf(m.half_alpha[src] * ch.ln_ratio);
    const float w = m.pol_m ? spec : m.sqrt_flux[src] * spec;
    const float4 M = m.pol_m ? m.pol_m[src] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ncomp = m.n_beam * m.n_feed * m.n_ax;
    if (m.beam_kind == 1) {
        const float a = w * expf(-m.gauss_c * azza.y * azza.y);
        out[0] = make_float2(a, 0.f);
        return fabsf(a);
    }
    // stencil in za (pole-reflected, clamped) and az (periodic)
    const bool cubic = m.interp == 0;
    const int nt = cubic ? 4 : 2;
    const float uz = azza.y / m.dza, ua = azza.x / m.daz;
    const float fz = floorf(uz), fa = floorf(ua);
    const float tz = uz - fz, ta = ua - fa;
    const int z0 = (int)fz - (cubic ? 1 : 0), a0 = (int)fa - (cubic ? 1 : 0);
    float wz[4], wa_[4];
    if (cubic) {
        wz[0] = keys(tz + 1.f); wz[1] = keys(tz); wz[2] = keys(1.f - tz); wz[3] = keys(2.f - tz);
        wa_[0] = keys(ta + 1.f); wa_[1] = keys(ta); wa_[2] = keys(1.f - ta); wa_[3] = keys(2.f - ta);
    } else {
        wz[0] = 1.f - tz; wz[1] = tz; wz[2] = wz[3] = 0.f;
        wa_[0] = 1.f - ta; wa_[1] = ta; wa_[2] = wa_[3] = 0.f;
    }
    int rows[4], shifts[4];
    float sg[4];
    const float pole_sign = m.n_ax == 2 ? -1.f : 1.f;
    for (int r = 0; r < nt; ++r) {
        int row = z0 + r, sh = 0;
        float g = 1.f;
        if (row < 0) { row = -row; sh = m.n_az / 2; g = pole_sign; }
        if (row > m.n_za - 1) row = m.n_za - 1;
        rows[r] = row; shifts[r] = sh; sg[r] = g * wz[r];
    }
    const long long plane = (long long)m.n_za * m.n_az;
    float mx = 0.f;
    float2 a_prev = make_float2(0.f, 0.f);
    for (int comp = 0; comp < ncomp; ++comp) {
        const float2* P = planes + ((long long)in.c * ncomp + comp) * plane;
        float re = 0.f, im = 0.f;
        for (int r = 0; r < nt; ++r) {
            const float2* rowp = P + (long long)rows[r] * m.n_az;
            float rr = 0.f, ri = 0.f;
            for (int q = 0; q < nt; ++q) {
                int col = (a0 + q + shifts[r]) % m.n_az;
                if (col < 0) col += m.n_az;
                const float2 v = rowp[col];
                rr = fmaf(wa_[q], v.x, rr);
                ri = fmaf(wa_[q], v.y, ri);
            }
            re = fmaf(sg[r], rr, re);
            im = fmaf(sg[r], ri, im);
        }
        if (!m.pol_m) {
            const float2 v = make_float2(w * re, w * im);
            out[(long long)comp * wa_pitch] = v;
            mx = fmaxf(mx, hypotf(v.x, v.y));
        } else if ((comp & 1) == 0) {  // axis 0 of a (beam, feed): wait for axis 1
            a_prev = make_float2(re, im);
        } else {
            float2 z0, z1;
            apply_sky_sqrt(a_prev, make_float2(re, im), M, w, z0, z1);
            out[(long long)(comp - 1) * wa_pitch] = z0;
            out[(long long)comp * wa_pitch] = z1;
            mx = fmaxf(mx, fmaxf(hypotf(z0.x, z0.y), hypotf(z1.x, z1.y)));
        }
    }
    return mx;
}

}  // namespace

cudaError_t launch_cull(const Model& m, const double* d_R, int n_times, LiveTables lt, int* d_counts,
                        int* d_offsets, int bpt, cudaStream_t st, long long* launches) {
    dim3 grid(bpt, n_times);
    k_cull_count<<<grid, kCullThreads, 0, st>>>(m, d_R, d_counts, bpt);
    k_cull_scan<<<n_times, 1024, 0, st>>>(d_counts, d_offsets, lt.n_live, bpt);
    k_cull_scatter<<<grid, kCullThreads, 0, st>>>(m, d_R, d_offsets, bpt, lt);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_beam_planes(const Model& m, const float2* d_grid, const Chan* d_chan, int n_chan,
                               float2* d_planes, cudaStream_t st, long long* launches) {
    const long long plane = (long long)m.n_za * m.n_az;
    dim3 grid((unsigned)((plane + 255) / 256), m.n_beam * m.n_feed * m.n_ax, n_chan);
    k_beam_planes<<<grid, 256, 0, st>>>(m, d_grid, d_chan, d_planes);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_wa(const Model& m, const float2* d_planes, const Chan* d_chan, const Inst* d_inst,
                      int inst0, int n_inst, LiveTables lt, float2* d_wa, long long wa_pitch, float* d_amax,
                      cudaStream_t st, long long* launches) {
    dim3 grid((unsigned)((lt.pitch + 127) / 128), n_inst);
    k_wa<<<grid, 128, 0, st>>>(m, d_planes, d_chan, d_inst, inst0, lt, d_wa, wa_pitch, d_amax);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
