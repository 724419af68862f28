// herk_fp32.cu -- Algorithm 2 step (v) of arXiv:2312.09763 (Sec. 3.1),
// V = Z Z^dagger (eq. "zz"), on the CUDA cores in FP32.
//
// Z is held as the real matrix U (rows 2(a n_feed + p) = Re, +1 = Im), so
// G = U U^T is symmetric and each complex entry of V is one 2 x 2 block:
//   Re V_ab = G[2a][2b] + G[2a+1][2b+1],   Im V_ab = G[2a+1][2b] - G[2a][2b+1].
// Only the lower triangle of 128 x 128 tiles of G is computed (a Hermitian
// rank-k update), and V is written in full (the upper triangle as the
// conjugate).  Each thread accumulates its 8 x 8 block in FP32 over at most
// `flush_k` sources, then adds that partial into a second FP32 running sum,
// which keeps the rounding error of long source sums near sqrt(K) ulp.
#include "common.cuh"

namespace mv {
namespace {

constexpr int BT = 128;  // output tile (rows and columns of G)
constexpr int BKF = 16;  // k step held in shared memory

__device__ __forceinline__ void tile_of(int p, int& ti, int& tj) {
    int i = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= p) ++i;
    while (i * (i + 1) / 2 > p) --i;
    ti = i;
    tj = p - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(256, 1)
k_herk_fp32(const Inst* __restrict__ inst, int inst0, LiveTables lt, int n_ax, const float* __restrict__ U,
            int rows, long long k_pitch, float2* __restrict__ V, int N, int flush_k) {
    __shared__ __align__(16) float As[2][BKF][BT];
    __shared__ __align__(16) float Bs[2][BKF][BT];
    const int slot = blockIdx.y;
    const Inst in = inst[inst0 + slot];
    int ti, tj;
    tile_of(blockIdx.x, ti, tj);
    const long long K = (long long)lt.n_live[in.t] * n_ax;
    const long long kpad = (K + kKPad - 1) / kKPad * kKPad;
    const float* Ub = U + (long long)slot * rows * k_pitch;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int rA = ti * BT, rB = tj * BT;

    float acc[8][8], run[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) { acc[i][j] = 0.f; run[i][j] = 0.f; }

    float4 pa[2], pb[2];
    auto gload = [&](long long k0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * 256;
            const int row = idx & (BT - 1), kq = (idx >> 7) * 4;
            const int ra = rA + row, rb = rB + row;
            pa[q] = ra < rows ? *reinterpret_cast<const float4*>(Ub + (long long)ra * k_pitch + k0 + kq)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            pb[q] = rb < rows ? *reinterpret_cast<const float4*>(Ub + (long long)rb * k_pitch + k0 + kq)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * 256;
            const int row = idx & (BT - 1), kq = (idx >> 7) * 4;
            As[buf][kq + 0][row] = pa[q].x; As[buf][kq + 1][row] = pa[q].y;
            As[buf][kq + 2][row] = pa[q].z; As[buf][kq + 3][row] = pa[q].w;
            Bs[buf][kq + 0][row] = pb[q].x; Bs[buf][kq + 1][row] = pb[q].y;
            Bs[buf][kq + 2][row] = pb[q].z; Bs[buf][kq + 3][row] = pb[q].w;
        }
    };

    const long long nsteps = kpad / BKF;
    if (nsteps > 0) { gload(0); sstore(0); }
    __syncthreads();
    const int steps_per_flush = flush_k / BKF;
    for (long long it = 0; it < nsteps; ++it) {
        const int buf = (int)(it & 1);
        if (it + 1 < nsteps) gload((it + 1) * BKF);
#pragma unroll
        for (int kk = 0; kk < BKF; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if ((it + 1) % steps_per_flush == 0 || it + 1 == nsteps) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) { run[i][j] += acc[i][j]; acc[i][j] = 0.f; }
        }
        if (it + 1 < nsteps) sstore(buf ^ 1);
        __syncthreads();
    }

    // epilogue: 2 x 2 blocks of G -> complex V entries (lower triangle + mirror)
    float2* Vb = V + in.v_off;
#pragma unroll
    for (int bi = 0; bi < 4; ++bi) {       // row pairs: 0,1 | 2,3 | 4,5 | 6,7 of the micro tile
#pragma unroll
        for (int bj = 0; bj < 4; ++bj) {
            const int li = 2 * bi, lj = 2 * bj;
            const int r = rA + (li < 4 ? ty * 4 + li : 64 + ty * 4 + (li - 4));
            const int c = rB + (lj < 4 ? tx * 4 + lj : 64 + tx * 4 + (lj - 4));
            const int a = r >> 1, b = c >> 1;
            if (a >= N || b >= N || a < b) continue;
            const float re = run[li][lj] + run[li + 1][lj + 1];
            const float im = run[li + 1][lj] - run[li][lj + 1];
            Vb[(long long)a * N + b] = make_float2(re, im);
            if (a != b) Vb[(long long)b * N + a] = make_float2(re, -im);
        }
    }
}

}  // namespace

cudaError_t launch_herk_fp32(const Inst* d_inst, int inst0, int n_inst, LiveTables lt, int n_ax, const float* d_u,
                             int rows, long long k_pitch, float2* d_v, int N, int flush_k, cudaStream_t st,
                             long long* launches) {
    const int T = (rows + BT - 1) / BT;
    if (flush_k < BKF || flush_k % BKF) flush_k = 256;
    dim3 grid(T * (T + 1) / 2, n_inst);
    k_herk_fp32<<<grid, 256, 0, st>>>(d_inst, inst0, lt, n_ax, d_u, rows, k_pitch, d_v, N, flush_k);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace mv
