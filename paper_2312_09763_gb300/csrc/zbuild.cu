// zbuild.cu -- Algorithm 2 steps (iii)-(iv) of arXiv:2312.09763 (Sec. 3.1):
// the antenna-based phase and the per-antenna matrix
// Z[(a,p),(s,k)] = sqrt(I_s) A^{pk}_{beta(a)}(s) exp(-2 pi i (nu/c) x_a . s_hat)
// of eq. "littlez" (Sec. 2.2), written as the real matrix U with interleaved
// rows 2(a n_feed + p) = Re Z, 2(a n_feed + p) + 1 = Im Z and columns
// s n_ax + k, so that V = Z Z^dagger becomes the real product U U^T.  The
// per-element arithmetic (fixed-point phase, recurrence, hi/lo split) is in
// zcore.cuh; this file holds the antenna phase table and the stand-alone
// Z-build kernel.
#include <cuda_fp16.h>

#include <algorithm>
#include "common.cuh"
#include "zcore.cuh"

namespace mv {
namespace {

using namespace zcore;

// Antenna factors of every wavenumber of a batch's groups: entry e of group
// gl is kappa0 (e = 0) and dkappa (e = 1) of an equally spaced group, or the
// wavenumber of its instance e otherwise.
__global__ void k_ant_phase(Model m, const Inst* __restrict__ inst, const Chan* __restrict__ chan,
                            const ZGroup* __restrict__ groups, int g_first, int n_phase, AntPhase* __restrict__ tab,
                            float* __restrict__ amax) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y, gl = blockIdx.z;
    const ZGroup g = groups[g_first + gl];
    if (amax && blockIdx.x == 0 && e == 0 && threadIdx.x == 0) {
        // one FP16 scale per group: every instance takes the group's max |WA|
        // (the Z build folds the scale into its cos/sin factors; the HERK
        // undoes it per instance from the same value)
        float mx = 0.f;
        for (int j = 0; j < g.n; ++j) mx = fmaxf(mx, amax[g.slot0 + j]);
        for (int j = 0; j < g.n; ++j) amax[g.slot0 + j] = mx;
    }
    if (a >= m.n_ant) return;
    double kap;
    if (g.uniform) {
        if (e >= 2) return;
        kap = e == 0 ? g.kappa0 : g.dkappa;
    } else {
        if (e >= g.n) return;
        kap = chan[inst[g.inst0 + e].c].kappa;
    }
    const double x[3] = {m.ant_e[a], m.ant_n[a], m.ant_u[a]};
    AntPhase p;
    unsigned long long nk = 0ull;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double y = kap * x[c];
        const long long Y = __double2ll_rn(y * 4294967296.0);  // 2^32
        p.yl[c] = (unsigned)Y;
        p.yh[c] = (int)(Y >> 32);
        p.yf[c] = (float)y;
        nk -= (unsigned long long)p.yl[c] << 31;
    }
    p.negk_lo = (unsigned)nk;
    p.negk_hi = (unsigned)(nk >> 32);
    p.pad = 0u;
    tab[((long long)gl * n_phase + e) * m.n_ant + a] = p;
}

// Grid-stride over the work items, so that the launch can be held to a fixed
// number of resident blocks per SM (room left for a concurrent HERK).  The
// FP16 scales of the item's instances go to shared memory once per item.
template <int PREC, int NAX, int NFD>
__global__ void __launch_bounds__(128, NAX * NFD > 1 ? 6 : 7)
k_zbuild(Model m, const Inst* __restrict__ inst, const ZGroup* __restrict__ groups, int g_first, LiveTables lt,
         const float2* __restrict__ wa, long long wa_pitch, const float* __restrict__ amax, void* u, void* ulo,
         int rows, long long k_pitch, int ant_per_block, const AntPhase* __restrict__ aph, int n_phase, int nx,
         int ny, long long n_items) {
    __shared__ float scale[kMaxBatch];
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int bx = (int)(item % nx);
        const long long rest = item / nx;
        const int by = (int)(rest % ny), bz = (int)(rest / ny);
        const ZGroup g = groups[g_first + bz];
        __syncthreads();  // the previous item's readers are done
        if (PREC == 2)
            for (int j = threadIdx.x; j < g.n; j += blockDim.x)
                scale[j] = ldexpf(1.f, fp16_scale_exp(amax[g.slot0 + j]));
        __syncthreads();
        zbuild_item<PREC, NAX, NFD>(m, inst, g, lt, wa, wa_pitch, scale, u, ulo, rows, k_pitch, ant_per_block,
                                    aph + (long long)bz * n_phase * m.n_ant, bx, by, blockDim.x, threadIdx.x);
    }
}

}  // namespace

cudaError_t launch_ant_phase(const Model& m, const Inst* d_inst, const Chan* d_chan, const ZGroup* d_groups,
                             int g_first, int n_groups, AntPhase* d_aph, int n_phase, float* d_amax, cudaStream_t st,
                             long long* launches) {
    if (!d_aph || n_phase < 2) return cudaErrorInvalidValue;
    k_ant_phase<<<dim3((unsigned)((m.n_ant + 127) / 128), (unsigned)n_phase, (unsigned)n_groups), 128, 0, st>>>(
        m, d_inst, d_chan, d_groups, g_first, n_phase, d_aph, d_amax);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_zbuild(const Model& m, const Inst* d_inst, const Chan* d_chan, const ZGroup* d_groups,
                          int g_first, int n_groups, LiveTables lt, const float2* d_wa, long long wa_pitch,
                          float* d_amax, void* d_u, void* d_u_lo, int prec, int rows, long long k_pitch,
                          int max_blocks, AntPhase* d_aph, int n_phase, cudaStream_t st, long long* launches) {
    if (!lt.sfix) return cudaErrorInvalidValue;
    cudaError_t e = launch_ant_phase(m, d_inst, d_chan, d_groups, g_first, n_groups, d_aph, n_phase,
                                     prec == 2 ? d_amax : nullptr, st, launches);
    if (e != cudaSuccess) return e;
    const int apb = 32;
    const int nx = (int)((lt.pitch / 2 + 127) / 128), ny = (m.n_ant + apb - 1) / apb;
    const long long n_items = (long long)nx * ny * n_groups;
    const long long grid = max_blocks > 0 ? std::min<long long>(n_items, max_blocks) : n_items;
#define MV_ZB(P, A, F) \
    k_zbuild<P, A, F><<<(unsigned)grid, 128, 0, st>>>(m, d_inst, d_groups, g_first, lt, d_wa, wa_pitch, d_amax, d_u, \
                                                      d_u_lo, rows, k_pitch, apb, d_aph, n_phase, nx, ny, n_items)
#define MV_ZB_P(A, F) \
    do { if (prec == 0) MV_ZB(0, A, F); else MV_ZB(2, A, F); } while (0)
    if (m.n_ax == 1) {
        if (m.n_feed == 1) MV_ZB_P(1, 1); else MV_ZB_P(1, 2);
    } else {
        if (m.n_feed == 1) MV_ZB_P(2, 1); else MV_ZB_P(2, 2);
    }
#undef MV_ZB_P
#undef MV_ZB
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
