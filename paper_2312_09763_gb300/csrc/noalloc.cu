// noalloc.cu -- mv_horizon_cull_static: the rotation + horizon-cut step with
// no device allocation.
//
// The regular path keeps the cut's per-block live counts and their prefix
// offsets in workspace that the context allocates.  Some callers cannot
// allocate device memory at the moment they need this step: hosts whose
// device memory all belongs to a framework's own pool (a cudaMalloc beside
// the pool can fail or fragment it), and latency-critical loops that cannot
// afford cudaMalloc's implicit device synchronisation.  This entry point
// serves them: its scratch is the file-scope array below, which every GPU
// that loads this library holds until the process exits.  The 3 x 3 rotation
// reaches the device as a kernel argument (copied at launch), so no host
// buffer has to outlive the call.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "matvis.h"
#include "common.cuh"

namespace {

// Maximum catalogue size per call: one scratch slot per 256 sources.
constexpr int kMaxCullBlocks = 8192;
constexpr long long kMaxStaticSources = (long long)kMaxCullBlocks * 256;  // 2,097,152

// Scratch: per-block live counts [0, kMaxCullBlocks) and their exclusive
// prefix offsets [kMaxCullBlocks, 2 kMaxCullBlocks), plus the 3 x 3 rotation.
// Every count and offset a call reads is written earlier in the same call,
// so nothing needs clearing; calls that overlap on the GPU race on it.
static __device__ __align__(256) int g_cull_scratch[2 * kMaxCullBlocks];
static __device__ __align__(256) double g_cull_rotation[9];

// Kernel argument carrying the rotation by value.
struct Rot9 {
    double r[9];
};

// Writes the rotation into g_cull_rotation (one thread per entry).
__global__ void k_put_rotation(Rot9 R) {
    if (threadIdx.x < 9) g_cull_rotation[threadIdx.x] = R.r[threadIdx.x];
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int* g_scratch_addr[kMaxDevices] = {};
double* g_rot_addr[kMaxDevices] = {};

mv_status fail(mv_status s, const char* m) {
    mv::set_last_error(m);
    return s;
}

}  // namespace

extern "C" mv_status mv_horizon_cull_static(int64_t n_src, const double* xeq_dev, double lst_rad,
                                            double latitude_rad, int32_t* live_idx_dev, double* enu_dev,
                                            float* azza_dev, int32_t* n_live_dev, void* stream) {
    mv::set_last_error("");
    if (n_src < 1 || n_src > kMaxStaticSources)
        return fail(MV_ERR_ARG, "mv_horizon_cull_static: n_src must be in [1, 2097152]");
    if (!xeq_dev || !live_idx_dev || !enu_dev || !azza_dev || !n_live_dev)
        return fail(MV_ERR_ARG, "mv_horizon_cull_static: NULL pointer argument");
    if (!std::isfinite(lst_rad) || !std::isfinite(latitude_rad))
        return fail(MV_ERR_ARG, "mv_horizon_cull_static: LST and latitude must be finite");
    if (std::fabs(latitude_rad) > 0.5 * mv::kPi)
        return fail(MV_ERR_ARG, "mv_horizon_cull_static: |latitude| must be <= pi/2");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(MV_ERR_CUDA, "mv_horizon_cull_static: no current CUDA device");
    int* scratch = nullptr;
    double* rot = nullptr;
    {
        // first call on a device: resolve the device addresses of the static arrays
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            void* q = nullptr;
            if (cudaGetSymbolAddress(&p, g_cull_scratch) != cudaSuccess ||
                cudaGetSymbolAddress(&q, g_cull_rotation) != cudaSuccess) {
                cudaGetLastError();
                return fail(MV_ERR_CUDA, "mv_horizon_cull_static: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[dev] = static_cast<int*>(p);
            g_rot_addr[dev] = static_cast<double*>(q);
        }
        scratch = g_scratch_addr[dev];
        rot = g_rot_addr[dev];
    }
    // eq. "rotation" of arXiv:2312.09763 with hour angle H = -LST (rows E, N, U)
    const double H = -lst_rad;
    const double sH = std::sin(H), cH = std::cos(H), sl = std::sin(latitude_rad), cl = std::cos(latitude_rad);
    const Rot9 R = {{sH, cH, 0.0, -sl * cH, sl * sH, cl, cl * cH, -cl * sH, sl}};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_put_rotation<<<1, 32, 0, st>>>(R);
    if (cudaGetLastError() != cudaSuccess) return fail(MV_ERR_CUDA, "mv_horizon_cull_static: rotation launch failed");
    mv::Model m{};
    m.n_src = n_src;
    m.xeq = xeq_dev;
    mv::LiveTables lt{};
    lt.e = enu_dev;
    lt.n = enu_dev + n_src;
    lt.u = enu_dev + 2 * n_src;
    lt.idx = live_idx_dev;
    lt.azza = reinterpret_cast<float2*>(azza_dev);
    lt.n_live = n_live_dev;
    lt.pitch = n_src;
    const int bpt = (int)((n_src + 255) / 256);
    long long launches = 0;
    cudaError_t e = mv::launch_cull(m, rot, 1, lt, scratch, scratch + kMaxCullBlocks, bpt, st, &launches);
    if (e != cudaSuccess) return fail(MV_ERR_CUDA, "mv_horizon_cull_static: launch failed");
    return MV_OK;
}
