// api.cu -- the extern "C" boundary (include/matvis.h) and the host runtime
// behind it: argument validation, the per-call plan (distinct times and
// channels, instance batches that share a time), workspace management, and
// the launch sequence of Algorithm 2 (arXiv:2312.09763, Sec. 3.1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "matvis.h"
#include "common.cuh"
#include "redund.h"

using namespace mv;

namespace {

thread_local std::string g_err;

mv_status fail(mv_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Configuration of the tensor-core HERK for one call.
struct HerkCfg {
    int bn = 256;     // tile columns
    int split = 1;    // source-axis split
    int flush = 4;    // k-blocks per TMEM flush
};

}  // namespace

void mv::set_last_error(const char* msg) { g_err = msg; }

struct mv_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mv_options opt{};
    Model model{};
    bool have_sky = false, have_ant = false, have_beam = false;
    double nu_ref = 150e6;
    double lat = 0.0;
    std::vector<int> h_bidx;
    std::vector<double> h_enu;  // [n_ant][3] (host copy, for the redundancy plan)
    double grid_nu0 = 0, grid_dnu = 0;
    // redundant-baseline expansion (mv_set_redundancy): the plan, the antenna
    // arrays in the cover's order, the group lookup and the tile lists
    RedPlan red;
    bool have_red = false;
    int red_nf = 0;  // feeds the plan was made for
    Buf red_e, red_n, red_u, red_b, red_uidx, red_tl[2];  // red_tl: 128- and 256-column tiles
    int red_ntl[2] = {0, 0};
    // model buffers
    std::vector<double> h_flux;  // I at nu_ref (host copy, for the polarised sky's coherency)
    Buf xeq, sqrt_flux, half_alpha, pol_m, ant_e, ant_n, ant_u, bidx, grid;
    // workspace
    Buf R, counts, offsets, le, ln, lu, lsfix, lseps, lidx, lazza, nlive, chan, inst, groups, planes, vdev, err, partial, sched;
    // per-batch workspace, double-buffered so that the beam evaluation and Z
    // build of one batch (on zstream) overlap the HERK of the previous one
    Buf wa[3], amax[3], u[2], ulo[2], aph[2];  // wa/amax: a third set when the beam runs two batches ahead
    cudaStream_t zstream = nullptr;
    cudaEvent_t ev_prep = nullptr, ev_zdone[2] = {nullptr, nullptr}, ev_hdone[2] = {nullptr, nullptr};
    // copies of each batch's V to pinned host memory, overlapping the next batches
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_vdone = nullptr, ev_cdone = nullptr;
    int n_sms = 148;
    // autotuned HERK configuration, valid for calls of the same shape
    struct Tuned {
        bool valid = false;
        int rows = 0, slots = 0, zprec = 0;
        HerkCfg cfg;
        bool fuse = true;  // the timed schedule: fused Z build, or separate Z-side launches
        double ms = 0;
    } tuned;
    // captured launch sequence of the last call shape
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<long long> graph_key;
    long long graph_launches = 0;
    long long launches = 0;
    std::vector<int> last_inst_t;
    // learned beam
    Surrogate* sur = nullptr;
    bool use_sur = false;
    mv_mlp_config sur_cfg{};
    // kernel timing
    bool profiling = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;          // recorded, not yet harvested
    std::vector<cudaEvent_t> pool;  // idle events
    long long prof_launches[MV_KERNEL_KINDS] = {0, 0, 0, 0};
    double prof_ms[MV_KERNEL_KINDS] = {0, 0, 0, 0};
};

namespace {

void buf_free(mv_ctx* c, Buf& b) {
    if (!b.p) return;
    if (c->opt.allocator.alloc && c->opt.allocator.free)
        c->opt.allocator.free(b.p, b.bytes, c->device, c->stream, c->opt.allocator.user);
    else
        cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Make `b` hold at least `bytes` (contents are not preserved on growth).
mv_status ensure(mv_ctx* c, Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (b.p && b.bytes >= bytes) return MV_OK;
    if (b.p) cudaDeviceSynchronize();  // work on any stream may still use it
    buf_free(c, b);
    void* p = nullptr;
    if (c->opt.allocator.alloc) {
        p = c->opt.allocator.alloc(bytes, c->device, c->stream, c->opt.allocator.user);
        if (!p) return fail(MV_ERR_OOM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MV_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = bytes;
    return MV_OK;
}

mv_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MV_OK;
    return fail(MV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// MV_DEBUG_SYNC=1: synchronise after every launch and report its status.
bool debug_sync() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("MV_DEBUG_SYNC");
        v = (e && *e && *e != '0') ? 1 : 0;
    }
    return v == 1;
}

cudaEvent_t ev_get(mv_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Event pair around one launch when timing is on (begin before, end after).
struct Timed {
    mv_ctx* c;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(mv_ctx* c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) {
        if (c->profiling) {
            a = ev_get(c);
            b = ev_get(c);
            cudaEventRecord(a, st);
        }
    }
    void end() {
        if (a) {
            cudaEventRecord(b, st);
            c->recs.push_back({kind, a, b});
            a = nullptr;
        }
    }
};

void harvest(mv_ctx* c) {
    for (auto& r : c->recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_ms[r.kind] += ms;
        c->prof_launches[r.kind] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
}

mv_status launched(cudaError_t e, const char* what, cudaStream_t st) {
    if (e == cudaSuccess && debug_sync()) {
        e = cudaStreamSynchronize(st);
        fprintf(stderr, "[matvis] %s: %s\n", what, cudaGetErrorString(e));
    }
    return cuda_check(e, what);
}

// Copy host data into a device buffer on the context stream (the host array
// may be released when this returns).
mv_status upload(mv_ctx* c, Buf& b, const void* h, size_t bytes, cudaStream_t st) {
    mv_status s = ensure(c, b, bytes);
    if (s) return s;
    if (bytes == 0) return MV_OK;
    return cuda_check(cudaMemcpyAsync(b.p, h, bytes, cudaMemcpyHostToDevice, st), "upload");
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// fn(begin, end, part) over [0, n) in up to 16 contiguous parts of at least
// 2^13 items on host threads; part numbers the parts from 0.
template <typename Fn>
void parallel_for(int64_t n, Fn fn) {
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(hw, n >> 13));
    if (parts <= 1) {
        fn((int64_t)0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(parts - 1);
    int k = 1;
    try {
        for (; k < parts; ++k) th.emplace_back(fn, n * k / parts, n * (k + 1) / parts, k);
    } catch (...) {  // no thread to be had: the rest on this one
        for (; k < parts; ++k) fn(n * k / parts, n * (k + 1) / parts, k);
    }
    fn((int64_t)0, n / parts, 0);
    for (auto& t : th) t.join();
}

// Smallest index i < n with !ok(i), or n.
template <typename Ok>
int64_t first_bad(int64_t n, Ok ok) {
    std::vector<int64_t> bad(16, n);
    parallel_for(n, [&](int64_t b, int64_t e, int part) {
        for (int64_t i = b; i < e; ++i)
            if (!ok(i)) { bad[part] = i; return; }
    });
    return *std::min_element(bad.begin(), bad.end());
}

bool finite_all(const double* p, int64_t n) {
    return first_bad(n, [p](int64_t i) { return std::isfinite(p[i]); }) == n;
}

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// Keys (1981) cubic-convolution weights (a = -1/2), FP64.
double keys_h(double x) {
    const double t = std::fabs(x);
    if (t <= 1.0) return (1.5 * t - 2.5) * t * t + 1.0;
    if (t < 2.0) return ((-0.5 * t + 2.5) * t - 4.0) * t + 2.0;
    return 0.0;
}

// One simulate call: distinct times and channels, instances, and batches of
// consecutive instances processed per launch (each batch a list of groups
// that share a time).
struct Plan {
    std::vector<double> lst;
    std::vector<double> nu;
    std::vector<Inst> inst;
    std::vector<ZGroup> groups;
    struct Batch { int inst0, n, g0, ng; };
    std::vector<Batch> batches;
    bool unique = false;  // one value per redundant group instead of the full V
};

// A group of consecutive instances [i0, i0+n) of one time: equally spaced
// channels get exact fixed-point phase stepping.
ZGroup make_group(const Plan& P, int i0, int n, int slot0) {
    ZGroup g{};
    g.inst0 = i0;
    g.n = n;
    g.slot0 = slot0;
    g.uniform = 0;
    const double nu0 = P.nu[P.inst[i0].c];
    if (n == 1) {
        g.uniform = 1;
        g.kappa0 = nu0 / kCLight;
        g.dkappa = 0.0;
        return g;
    }
    const double nu1 = P.nu[P.inst[i0 + n - 1].c];
    const double dnu = (nu1 - nu0) / (n - 1);
    bool uni = true;
    for (int j = 0; j < n && uni; ++j) {
        const double want = nu0 + j * dnu;
        if (std::fabs(P.nu[P.inst[i0 + j].c] - want) > 1e-12 * std::fabs(want)) uni = false;
    }
    if (uni) {
        g.uniform = 1;
        g.kappa0 = nu0 / kCLight;
        g.dkappa = dnu / kCLight;
    }
    return g;
}

int auto_batch(mv_ctx* c, long long slot_bytes) {
    if (c->opt.max_batch > 0) return std::min(c->opt.max_batch, kMaxBatch);
    const long long budget = 20ll << 30;  // workspace for the Z planes
    long long b = budget / std::max(slot_bytes, 1ll);
    return (int)std::max(1ll, std::min(b, 64ll));
}

// Workspace of one instance slot: the Z planes plus its beam x sqrt(I) table.
long long slot_bytes_of(mv_ctx* c) {
    const Model& m = c->model;
    const long long N = (long long)m.n_feed * m.n_ant;
    const long long src = std::max<long long>(m.n_src, 1);
    const long long ncomp = (long long)std::max(m.n_beam, 1) * std::max(m.n_feed, 1) * std::max(m.n_ax, 1);
    return 4ll * 2 * N * round_up((long long)m.n_ax * src, kKPad) + 8ll * ncomp * round_up(src, kKPad);
}

constexpr int kZGroup = 16;  // the fused Z build keeps a group's FP16 scales in 16 floats per warp
static_assert(kZGroup <= 16, "Z groups of at most 16 instances");

// Every (LST, channel) pair; batches are up to B channels of one LST.
void plan_grid(mv_ctx* c, int n_t, const double* lst, int n_nu, const double* nu, Plan& P) {
    P.lst.assign(lst, lst + n_t);
    P.nu.assign(nu, nu + n_nu);
    const long long N = (long long)c->model.n_feed * c->model.n_ant;
    for (int t = 0; t < n_t; ++t)
        for (int f = 0; f < n_nu; ++f) P.inst.push_back(Inst{t, f, ((long long)t * n_nu + f) * N * N});
    const int B = auto_batch(c, slot_bytes_of(c));
    for (int t = 0; t < n_t; ++t)
        for (int f0 = 0; f0 < n_nu; f0 += B) {
            const int n = std::min(B, n_nu - f0);
            const int i0 = t * n_nu + f0;
            // Z build groups of at most kZGroup channels: one launch covers the
            // batch, but its blocks work through the groups in order, so the
            // slots written at any time (and their pages) stay few
            Plan::Batch b{i0, n, (int)P.groups.size(), 0};
            for (int c0 = 0; c0 < n; c0 += kZGroup, ++b.ng)
                P.groups.push_back(make_group(P, i0 + c0, std::min(kZGroup, n - c0), c0));
            P.batches.push_back(b);
        }
}

// Explicit (LST, frequency) pairs; batches of up to B pairs, one group each.
void plan_pairs(mv_ctx* c, int n_pairs, const double* lst, const double* nu, Plan& P) {
    P.lst.assign(lst, lst + n_pairs);
    P.nu.assign(nu, nu + n_pairs);
    const long long N = (long long)c->model.n_feed * c->model.n_ant;
    for (int i = 0; i < n_pairs; ++i) P.inst.push_back(Inst{i, i, (long long)i * N * N});
    const int B = auto_batch(c, slot_bytes_of(c));
    for (int i0 = 0; i0 < n_pairs; i0 += B) {
        const int n = std::min(B, n_pairs - i0);
        Plan::Batch b{i0, n, (int)P.groups.size(), n};
        for (int j = 0; j < n; ++j) P.groups.push_back(make_group(P, i0 + j, 1, j));
        P.batches.push_back(b);
    }
}

// Everything one simulate call needs on the device, after validation and uploads.
struct Prepared {
    int n_times = 0, n_chan = 0, n_inst = 0;
    int N = 0, rows = 0, bpt = 0, ncomp = 0, max_slots = 0, zprec = 0;
    int nbuf = 1;  // workspace sets in use (2: Z side and HERK overlap, or fused Z build)
    bool fuse = false;  // the HERK of batch b builds the Z planes of batch b + 1
    bool ahead = false;  // (fused) the beam of batch b + 2 runs on zstream beside the HERK of batch b
    int n_phase = 2;  // AntPhase entries per group
    const Plan* plan = nullptr;
    std::vector<int> h_nlive;  // live counts on the host (learned-beam calls only)
    long long pitch = 0, k_pitch = 0;
    LiveTables lt{};
    float2* Vout = nullptr;
    float2* Vhost = nullptr;  // page-locked host V (copied per batch on cstream), or NULL
    size_t v_bytes = 0;
    long long per_inst = 0;  // output values per instance: N^2, or n_unique n_feed^2
    HerkOut ho{};             // unique output: group lookup and tile lists (ho.tl set per tile width)
};

// Heuristic HERK configuration: wide tiles unless the matrix is narrow; a
// split giving the persistent grid about 16 units per SM while each unit keeps
// at least 32 k-blocks of the expected live count (half the catalogue).
HerkCfg heuristic_cfg(mv_ctx* c, const Prepared& p) {
    HerkCfg h;
    h.bn = c->opt.herk_tile_n == 128 || c->opt.herk_tile_n == 256 ? c->opt.herk_tile_n
                                                                   : (p.fuse || p.rows <= 128 ? 128 : 256);
    h.flush = c->opt.herk_flush_kblocks > 0 ? c->opt.herk_flush_kblocks : 4;
    const int base = herk_tc_units(p.rows, p.max_slots, 1, h.bn);
    const long long est_kb = std::max(1ll, ((long long)c->model.n_ax * c->model.n_src / 2 + 63) / 64);
    h.split = c->opt.herk_split > 0
                  ? c->opt.herk_split
                  : (int)std::max(1ll, std::min((long long)(16 * c->n_sms + base - 1) / base, est_kb / 32));
    return h;
}

bool tuned_for(const mv_ctx* c, const Prepared& p) {
    return c->tuned.valid && c->tuned.rows == p.rows && c->tuned.slots == p.max_slots && c->tuned.zprec == p.zprec;
}

HerkCfg chosen_cfg(mv_ctx* c, const Prepared& p) {
    if (p.ho.uidx) {
        // the redundant-group cover: its own tile count, 128 columns unless
        // forced (its narrow blocks leave a 256-column tiling short of MMA work
        // per ring stage: 141 against 112 ms per step on the 350-antenna array)
        HerkCfg h;
        h.bn = c->opt.herk_tile_n == 256 ? 256 : 128;
        h.flush = c->opt.herk_flush_kblocks > 0 ? c->opt.herk_flush_kblocks : 16;
        const int n_tl = c->red.kind == 0 ? herk_tc_units(p.rows, 1, 1, h.bn) : c->red_ntl[h.bn == 128 ? 0 : 1];
        const long long base = std::max(1ll, (long long)n_tl * p.max_slots);
        const long long est_kb = std::max(1ll, ((long long)c->model.n_ax * c->model.n_src / 2 + 63) / 64);
        h.split = c->opt.herk_split > 0
                      ? c->opt.herk_split
                      : (int)std::max(1ll, std::min((4ll * c->n_sms + base - 1) / base, est_kb / 32));
        return h;
    }
    if (tuned_for(c, p)) return c->tuned.cfg;
    return heuristic_cfg(c, p);
}

mv_status prepare(mv_ctx* c, Plan& P, mv_precision prec, void* V, int V_on_device, cudaStream_t st, Prepared& out) {
    Model& m = c->model;
    if (!c->have_sky || !c->have_ant || !c->have_beam)
        return fail(MV_ERR_STATE, "simulate needs init_sky, set_antennas and a beam first");
    if (m.pol_m && m.n_ax != 2) return fail(MV_ERR_STATE, "a polarised sky needs a two-axis beam");
    if (prec == 1)
        return fail(MV_ERR_ARG, "precision 1 (BF16 hi + lo) is not offered: 16 significant bits per entry of Z "
                                "cannot meet the 1e-5 bound; use MV_PREC_FP16X3");
    if (prec != MV_PREC_FP32 && prec != MV_PREC_FP16X3)
        return fail(MV_ERR_ARG, "unknown precision %d", (int)prec);
    if (!V) return fail(MV_ERR_ARG, "V is NULL");
    if (prec != MV_PREC_FP32 && !herk_tc_available())
        return fail(MV_ERR_UNSUPPORTED, "tensor-map encoding unavailable in this driver");
    for (int b : c->h_bidx)
        if (b >= m.n_beam) return fail(MV_ERR_ARG, "antenna beam index %d >= n_beam %d", b, m.n_beam);
    Prepared& p = out;
    p.plan = &P;
    p.n_times = (int)P.lst.size();
    p.n_chan = (int)P.nu.size();
    p.n_inst = (int)P.inst.size();
    p.zprec = prec == MV_PREC_FP32 ? 0 : 2;
    if (p.n_inst == 0) return MV_OK;

    // channel table
    std::vector<Chan> chan(p.n_chan);
    for (int i = 0; i < p.n_chan; ++i) {
        const double nu = P.nu[i];
        if (!(std::isfinite(nu) && nu > 0)) return fail(MV_ERR_ARG, "frequency %d is not positive and finite", i);
        chan[i].kappa = nu / kCLight;
        chan[i].ln_ratio = (float)std::log(nu / c->nu_ref);
        chan[i].m0 = 0;
        for (int j = 0; j < 4; ++j) chan[i].w[j] = 0.f;
        if (m.beam_kind == 2) {
            const double u = (nu - c->grid_nu0) / c->grid_dnu;
            const double f = std::floor(u);
            const double t = u - f;
            const int m0 = (int)f - 1;
            if (m0 < 0 || m0 + 3 > m.n_nu - 1)
                return fail(MV_ERR_ARG, "frequency %.9g Hz outside the beam grid's cubic margin", nu);
            chan[i].m0 = m0;
            chan[i].w[0] = (float)keys_h(t + 1.0);
            chan[i].w[1] = (float)keys_h(t);
            chan[i].w[2] = (float)keys_h(1.0 - t);
            chan[i].w[3] = (float)keys_h(2.0 - t);
        }
    }
    // R(t): eq. "rotation" with hour angle H = -LST; rows East, North, Up
    std::vector<double> R(9 * (size_t)p.n_times);
    const double sl = std::sin(c->lat), cl = std::cos(c->lat);
    for (int t = 0; t < p.n_times; ++t) {
        if (!std::isfinite(P.lst[t])) return fail(MV_ERR_ARG, "LST %d is not finite", t);
        const double H = -P.lst[t];
        const double sH = std::sin(H), cH = std::cos(H);
        double* r = &R[9 * (size_t)t];
        r[0] = sH;        r[1] = cH;        r[2] = 0.0;
        r[3] = -sl * cH;  r[4] = sl * sH;   r[5] = cl;
        r[6] = cl * cH;   r[7] = -cl * sH;  r[8] = sl;
    }

    // sizes
    p.N = m.n_feed * m.n_ant;
    p.rows = 2 * p.N;
    p.pitch = round_up(m.n_src, kKPad);
    p.k_pitch = round_up((long long)m.n_ax * m.n_src, kKPad);
    p.bpt = (int)((m.n_src + 255) / 256);
    p.ncomp = m.n_beam * m.n_feed * m.n_ax;
    p.max_slots = 0;
    for (auto& b : P.batches) p.max_slots = std::max(p.max_slots, b.n);
    p.per_inst = P.unique ? (long long)c->red.rep_a.size() * m.n_feed * m.n_feed : (long long)p.N * p.N;
    p.ho = HerkOut{};
    if (P.unique) {
        if (!c->have_red) return fail(MV_ERR_STATE, "no redundancy plan (mv_set_redundancy)");
        if (p.zprec == 0) return fail(MV_ERR_ARG, "the redundant-group output needs a tensor-core precision");
        p.ho.uidx = (const int*)c->red_uidx.p;
        p.ho.n_ant = m.n_ant;
        p.ho.n_feed = m.n_feed;
    }
    const int n_times = p.n_times, max_slots = p.max_slots;
    const long long pitch = p.pitch;

    mv_status s;
    if ((s = upload(c, c->R, R.data(), R.size() * sizeof(double), st))) return s;
    if ((s = upload(c, c->chan, chan.data(), chan.size() * sizeof(Chan), st))) return s;
    if ((s = upload(c, c->inst, P.inst.data(), P.inst.size() * sizeof(Inst), st))) return s;
    if ((s = upload(c, c->groups, P.groups.data(), P.groups.size() * sizeof(ZGroup), st))) return s;
    if ((s = ensure(c, c->counts, sizeof(int) * (size_t)p.bpt * n_times))) return s;
    if ((s = ensure(c, c->offsets, sizeof(int) * (size_t)p.bpt * n_times))) return s;
    if ((s = ensure(c, c->le, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->ln, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lu, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lsfix, sizeof(unsigned) * 3 * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lseps, sizeof(float) * 3 * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lidx, sizeof(int) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lazza, sizeof(float2) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->nlive, sizeof(int) * (size_t)n_times))) return s;
    // the fused schedule unless the autotuner timed the separate one faster
    // for calls of this shape; for the redundant-group output only when the
    // cover is the whole triangle: a cover of fewer tiles leaves the HERK too
    // short to hide the next batch's Z build (350-antenna array, 9 of 21
    // tiles: 250 ms per step fused against 210 ms separate)
    p.fuse = c->opt.fuse_zbuild && p.zprec != 0 && P.batches.size() > 1 &&
             herk_tc_fusable(128, p.zprec, m.n_ax, m.n_feed) && !(tuned_for(c, p) && !c->tuned.fuse) &&
             (!P.unique || c->red.kind == 0);
    p.nbuf = (P.batches.size() > 1 && (c->opt.overlap_batches || p.fuse)) ? 2 : 1;
    // antenna phase factors: per batch, groups x wavenumbers per group x antennas
    p.n_phase = 2;
    int max_groups = 1;
    for (auto& b : P.batches) {
        max_groups = std::max(max_groups, b.ng);
        for (int gi = b.g0; gi < b.g0 + b.ng; ++gi)
            if (!P.groups[gi].uniform) p.n_phase = std::max(p.n_phase, P.groups[gi].n);
    }
    // the beam two batches ahead (fused, not the learned beam, whose kernel needs whole SMs)
    p.ahead = p.fuse && !c->use_sur && P.batches.size() > 2;
    for (int k = 0; k < (p.ahead ? 3 : p.nbuf); ++k) {
        if ((s = ensure(c, c->wa[k], sizeof(float2) * (size_t)max_slots * p.ncomp * pitch))) return s;
        if ((s = ensure(c, c->amax[k], sizeof(float) * (size_t)max_slots))) return s;
    }
    for (int k = 0; k < p.nbuf; ++k)
        if ((s = ensure(c, c->aph[k], sizeof(AntPhase) * (size_t)max_groups * p.n_phase * m.n_ant))) return s;
    if ((s = ensure(c, c->sched, sizeof(int) * (size_t)(max_slots + 8)))) return s;
    const size_t plane_elems = (size_t)p.rows * p.k_pitch * max_slots;
    for (int k = 0; k < p.nbuf; ++k) {
        if (p.zprec == 0) {
            if ((s = ensure(c, c->u[k], sizeof(float) * plane_elems))) return s;
        } else {
            if ((s = ensure(c, c->u[k], 2 * plane_elems))) return s;
            if ((s = ensure(c, c->ulo[k], 2 * plane_elems))) return s;
        }
    }
    if (p.zprec != 0) {
        // partial tiles for the largest split any configuration may use
        const HerkCfg h = chosen_cfg(c, p);
        size_t units = (size_t)herk_tc_units(p.rows, max_slots, h.split, h.bn);
        if (P.unique) units = std::max(units, (size_t)c->red_ntl[h.bn == 128 ? 0 : 1] * max_slots * h.split);
        const size_t need = sizeof(float) * 128 * h.bn * units;
        if (h.split > 1 && (s = ensure(c, c->partial, need))) return s;
    }
    if (m.beam_kind == 2 &&
        (s = ensure(c, c->planes, sizeof(float2) * (size_t)p.n_chan * p.ncomp * m.n_za * m.n_az)))
        return s;
    p.Vout = static_cast<float2*>(V);
    p.v_bytes = sizeof(float2) * (size_t)p.n_inst * p.per_inst;
    p.Vhost = nullptr;
    if (!V_on_device) {
        if ((s = ensure(c, c->vdev, p.v_bytes))) return s;
        p.Vout = static_cast<float2*>(c->vdev.p);
        // page-locked host output: each batch's V is copied as soon as its HERK ends
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, V) == cudaSuccess && pa.type == cudaMemoryTypeHost)
            p.Vhost = static_cast<float2*>(V);
        cudaGetLastError();
    }
    LiveTables& lt = p.lt;
    lt.e = (double*)c->le.p;
    lt.n = (double*)c->ln.p;
    lt.u = (double*)c->lu.p;
    lt.sfix = (unsigned*)c->lsfix.p;
    lt.seps = (float*)c->lseps.p;
    lt.idx = (int*)c->lidx.p;
    lt.azza = (float2*)c->lazza.p;
    lt.n_live = (int*)c->nlive.p;
    lt.pitch = pitch;
    return MV_OK;
}

// HERK of one batch with configuration h.
// (k: the workspace set of the batch's U planes; kw: of its WA and amax, k if < 0)
cudaError_t enqueue_herk(mv_ctx* c, const Prepared& p, const Plan::Batch& b, const HerkCfg& h, int k,
                         cudaStream_t st, long long* L, const ZJob* zj = nullptr, int kw = -1) {
    if (kw < 0) kw = k;
    const Inst* d_inst = (const Inst*)c->inst.p;
    HerkOut ho = p.ho;
    if (ho.uidx) {
        const int w = h.bn == 128 ? 0 : 1;
        ho.tl = c->red.kind == 0 ? nullptr : (const TileDesc*)c->red_tl[w].p;
        ho.n_tl = c->red.kind == 0 ? 0 : c->red_ntl[w];
    }
    if (p.zprec == 0)
        return launch_herk_fp32(d_inst, b.inst0, b.n, p.lt, c->model.n_ax, (const float*)c->u[k].p, p.rows,
                                p.k_pitch, p.Vout, p.N, 256, st, L);
    return launch_herk_tc(d_inst, b.inst0, b.n, p.lt, c->model.n_ax, (const __nv_bfloat16*)c->u[k].p,
                          (const __nv_bfloat16*)c->ulo[k].p, p.rows, p.k_pitch, p.max_slots, p.zprec == 2 ? 1 : 0,
                          (const float*)c->amax[kw].p, p.Vout, p.N, h.flush, h.split, h.bn, c->n_sms, (int*)c->sched.p,
                          (float*)c->partial.p, (int*)c->err.p, zj, p.zprec, p.ho.uidx ? &ho : nullptr, st, L);
}

// The Z build of batch b into workspace set k, for the HERK of the batch before.
ZJob make_zjob(mv_ctx* c, const Prepared& p, const Plan::Batch& b, int k, int kw = -1) {
    if (kw < 0) kw = k;
    ZJob z{};
    z.m = c->model;
    z.inst = (const Inst*)c->inst.p;
    z.groups = (const ZGroup*)c->groups.p;
    z.g_first = b.g0;
    z.n_groups = b.ng;
    z.lt = p.lt;
    z.wa = (const float2*)c->wa[kw].p;
    z.wa_pitch = p.pitch;
    z.amax = (const float*)c->amax[kw].p;
    z.u = c->u[k].p;
    z.ulo = c->ulo[k].p;
    z.rows = p.rows;
    z.k_pitch = p.k_pitch;
    z.aph = (const AntPhase*)c->aph[k].p;
    z.n_phase = p.n_phase;
    return z;
}

// Beam evaluation of one batch into workspace set k.
mv_status enqueue_wa(mv_ctx* c, const Prepared& p, const Plan::Batch& b, int k, cudaStream_t st, long long* L) {
    mv_status s;
    const Model& m = c->model;
    const Inst* d_inst = (const Inst*)c->inst.p;
    if ((s = cuda_check(cudaMemsetAsync(c->amax[k].p, 0, sizeof(float) * b.n, st), "amax reset"))) return s;
    Timed tw(c, MV_KERNEL_BEAM, st);
    cudaError_t e;
    if (c->use_sur)
        e = surrogate_wa(c->sur, m, p.plan->inst, b.inst0, b.n, p.h_nlive, p.plan->nu, c->nu_ref, p.lt,
                         (float2*)c->wa[k].p, p.pitch, (float*)c->amax[k].p, (int*)c->err.p, c->n_sms, st, L);
    else
        e = launch_wa(m, (const float2*)c->planes.p, (const Chan*)c->chan.p, d_inst, b.inst0, b.n, p.lt,
                      (float2*)c->wa[k].p, p.pitch, (float*)c->amax[k].p, st, L);
    tw.end();
    return launched(e, "beam evaluation", st);
}

// Antenna phase table of one batch into workspace set k (fused Z build).
mv_status enqueue_ant_phase(mv_ctx* c, const Prepared& p, const Plan::Batch& b, int k, cudaStream_t st,
                            long long* L, int kw = -1) {
    if (kw < 0) kw = k;
    Timed tz(c, MV_KERNEL_ZBUILD, st);
    cudaError_t e = launch_ant_phase(c->model, (const Inst*)c->inst.p, (const Chan*)c->chan.p,
                                     (const ZGroup*)c->groups.p, b.g0, b.ng, (AntPhase*)c->aph[k].p, p.n_phase,
                                     p.zprec == 2 ? (float*)c->amax[kw].p : nullptr, st, L);
    tz.end();
    return launched(e, "phase table", st);
}

// Beam evaluation and Z build of one batch.
mv_status enqueue_zside(mv_ctx* c, const Prepared& p, const Plan::Batch& b, int k, cudaStream_t st, long long* L) {
    mv_status s;
    const Model& m = c->model;
    const Inst* d_inst = (const Inst*)c->inst.p;
    if ((s = enqueue_wa(c, p, b, k, st, L))) return s;
    Timed tz(c, MV_KERNEL_ZBUILD, st);
    cudaError_t e = launch_zbuild(m, d_inst, (const Chan*)c->chan.p, (const ZGroup*)c->groups.p, b.g0, b.ng, p.lt,
                      (const float2*)c->wa[k].p, p.pitch, (float*)c->amax[k].p, c->u[k].p, c->ulo[k].p,
                      p.zprec, p.rows, p.k_pitch, p.nbuf == 2 && !p.fuse ? 4 * c->n_sms : 0, (AntPhase*)c->aph[k].p,
                      p.n_phase, st, L);
    tz.end();
    return launched(e, "Z build", st);
}

// The whole launch sequence of a call: cull, beam planes, then per batch
// beam evaluation, Z build and HERK.
mv_status enqueue_all(mv_ctx* c, Plan& P, Prepared& p, const HerkCfg& h, cudaStream_t st, long long* L) {
    mv_status s;
    const Model& m = c->model;
    // page-locked host output: the batch's V (contiguous instances) goes to the
    // host on cstream once the HERK queued before this point on st is done
    auto copy_out = [&](const Plan::Batch& b) -> mv_status {
        if (!p.Vhost) return MV_OK;
        const long long off = P.inst[b.inst0].v_off;
        const size_t bytes = sizeof(float2) * (size_t)b.n * p.per_inst;
        mv_status s2;
        if ((s2 = cuda_check(cudaEventRecord(c->ev_vdone, st), "event"))) return s2;
        if ((s2 = cuda_check(cudaStreamWaitEvent(c->cstream, c->ev_vdone, 0), "event wait"))) return s2;
        return cuda_check(cudaMemcpyAsync(p.Vhost + off, p.Vout + off, bytes, cudaMemcpyDeviceToHost, c->cstream),
                          "copy V to host");
    };
    // st waits for the copies (they also join a stream capture)
    auto join_copies = [&]() -> mv_status {
        if (!p.Vhost) return MV_OK;
        mv_status s2;
        if ((s2 = cuda_check(cudaEventRecord(c->ev_cdone, c->cstream), "event"))) return s2;
        return cuda_check(cudaStreamWaitEvent(st, c->ev_cdone, 0), "event wait");
    };
    Timed tc0(c, MV_KERNEL_CULL, st);
    cudaError_t e = launch_cull(m, (const double*)c->R.p, p.n_times, p.lt, (int*)c->counts.p, (int*)c->offsets.p,
                                p.bpt, st, L);
    tc0.end();
    if ((s = launched(e, "cull", st))) return s;
    if (c->use_sur) {
        // the network's row count per instance is n_beam x live count: read them
        p.h_nlive.assign(p.n_times, 0);
        if ((s = cuda_check(cudaMemcpyAsync(p.h_nlive.data(), p.lt.n_live, sizeof(int) * p.n_times,
                                            cudaMemcpyDeviceToHost, st), "live counts")))
            return s;
        if ((s = cuda_check(cudaStreamSynchronize(st), "synchronize"))) return s;
    } else if (m.beam_kind == 2) {
        Timed tb(c, MV_KERNEL_BEAM, st);
        e = launch_beam_planes(m, (const float2*)c->grid.p, (const Chan*)c->chan.p, p.n_chan, (float2*)c->planes.p,
                               st, L);
        tb.end();
        if ((s = launched(e, "beam planes", st))) return s;
    }
    if (p.fuse) {
        // batch 0 alone; then the HERK launch of batch b also builds the Z
        // planes of batch b + 1 (its beam evaluation and phase table first)
        // into the other workspace set.  With p.ahead the beam evaluation and
        // phase table of batch b + 2 run on zstream beside the HERK of batch b
        // (WA and amax in three sets, batch mod 3; U planes and phase tables in
        // two, batch mod 2): zstream waits for the HERK of batch b - 1, the last
        // reader of the sets it overwrites, and the HERK of batch b + 1 waits
        // for them.
        const size_t B = P.batches.size();
        auto wset = [&](size_t i) { return p.ahead ? (int)(i % 3) : (int)(i & 1); };
        cudaStream_t zs = c->zstream;
        if ((s = enqueue_zside(c, p, P.batches[0], 0, st, L))) return s;
        if (p.ahead) {
            if ((s = enqueue_wa(c, p, P.batches[1], wset(1), st, L))) return s;
            if ((s = enqueue_ant_phase(c, p, P.batches[1], 1, st, L, wset(1)))) return s;
            if ((s = cuda_check(cudaEventRecord(c->ev_prep, st), "event"))) return s;
            if ((s = cuda_check(cudaStreamWaitEvent(zs, c->ev_prep, 0), "event wait"))) return s;
        }
        for (size_t i = 0; i < B; ++i) {
            const int k = (int)(i & 1);
            ZJob zj{};
            const bool next = i + 1 < B;
            if (p.ahead) {
                if (i + 2 < B) {
                    if (i >= 1 && (s = cuda_check(cudaStreamWaitEvent(zs, c->ev_hdone[(i - 1) & 1], 0), "event wait")))
                        return s;
                    const auto& b2 = P.batches[i + 2];
                    if ((s = enqueue_wa(c, p, b2, wset(i + 2), zs, L))) return s;
                    if ((s = enqueue_ant_phase(c, p, b2, (int)((i + 2) & 1), zs, L, wset(i + 2)))) return s;
                    if ((s = cuda_check(cudaEventRecord(c->ev_zdone[(i + 2) & 1], zs), "event"))) return s;
                }
                if (i >= 1 && next &&
                    (s = cuda_check(cudaStreamWaitEvent(st, c->ev_zdone[(i + 1) & 1], 0), "event wait")))
                    return s;
            } else if (next) {
                const auto& bn = P.batches[i + 1];
                if ((s = enqueue_wa(c, p, bn, k ^ 1, st, L))) return s;
                if ((s = enqueue_ant_phase(c, p, bn, k ^ 1, st, L))) return s;
            }
            if (next) zj = make_zjob(c, p, P.batches[i + 1], k ^ 1, wset(i + 1));
            Timed th(c, MV_KERNEL_HERK, st);
            e = enqueue_herk(c, p, P.batches[i], h, k, st, L, next ? &zj : nullptr, wset(i));
            th.end();
            if ((s = launched(e, "HERK tc", st))) return s;
            if (p.ahead && (s = cuda_check(cudaEventRecord(c->ev_hdone[k], st), "event"))) return s;
            if ((s = copy_out(P.batches[i]))) return s;
        }
        if (p.ahead) {  // zstream rejoins st (it also joins a stream capture)
            if ((s = cuda_check(cudaEventRecord(c->ev_prep, zs), "event"))) return s;
            if ((s = cuda_check(cudaStreamWaitEvent(st, c->ev_prep, 0), "event wait"))) return s;
        }
        return join_copies();
    }
    if (p.nbuf == 1) {
        for (const auto& b : P.batches) {
            if ((s = enqueue_zside(c, p, b, 0, st, L))) return s;
            Timed th(c, MV_KERNEL_HERK, st);
            e = enqueue_herk(c, p, b, h, 0, st, L);
            th.end();
            if ((s = launched(e, p.zprec == 0 ? "HERK fp32" : "HERK tc", st))) return s;
            if ((s = copy_out(b))) return s;
        }
        return join_copies();
    }
    // Two workspace sets: batch b builds Z into set b % 2 on zstream while the
    // HERK of batch b - 1 reads the other set on st.  zstream first waits for
    // everything already queued on st (earlier calls included); before reusing
    // a set it waits for the HERK that read it.
    cudaStream_t zs = c->zstream;
    if ((s = cuda_check(cudaEventRecord(c->ev_prep, st), "event"))) return s;
    if ((s = cuda_check(cudaStreamWaitEvent(zs, c->ev_prep, 0), "event wait"))) return s;
    for (size_t i = 0; i < P.batches.size(); ++i) {
        const auto& b = P.batches[i];
        const int k = (int)(i & 1);
        if (i >= 2 && (s = cuda_check(cudaStreamWaitEvent(zs, c->ev_hdone[k], 0), "event wait"))) return s;
        if ((s = enqueue_zside(c, p, b, k, zs, L))) return s;
        if ((s = cuda_check(cudaEventRecord(c->ev_zdone[k], zs), "event"))) return s;
        if ((s = cuda_check(cudaStreamWaitEvent(st, c->ev_zdone[k], 0), "event wait"))) return s;
        Timed th(c, MV_KERNEL_HERK, st);
        e = enqueue_herk(c, p, b, h, k, st, L);
        th.end();
        if ((s = launched(e, p.zprec == 0 ? "HERK fp32" : "HERK tc", st))) return s;
        if ((s = cuda_check(cudaEventRecord(c->ev_hdone[k], st), "event"))) return s;
        if ((s = copy_out(b))) return s;
    }
    return join_copies();
}

// Key of a captured launch sequence: every value its kernel arguments depend on.
// The model goes in by value (its pointers, sizes and beam scalars): set-up
// calls that refill the same buffers with data of the same shape keep the
// captured sequence, which reads the new data.
std::vector<long long> graph_key(mv_ctx* c, const Plan& P, const Prepared& p, const HerkCfg& h) {
    const Model& m = c->model;
    auto bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, sizeof u);
        return (long long)u;
    };
    std::vector<long long> k = {p.n_times, p.n_chan, p.n_inst, p.zprec, p.rows, p.max_slots, p.pitch, p.k_pitch, p.nbuf,
                                p.fuse, h.bn, h.split, h.flush, (long long)(uintptr_t)p.Vout,
                                (long long)(uintptr_t)p.Vhost, P.unique ? 1 : 0, p.per_inst, c->red.kind,
                                c->red_ntl[0], c->red_ntl[1],
                                m.n_src, (long long)(uintptr_t)m.xeq, (long long)(uintptr_t)m.sqrt_flux,
                                (long long)(uintptr_t)m.half_alpha, (long long)(uintptr_t)m.pol_m, m.n_ant,
                                (long long)(uintptr_t)m.ant_e, (long long)(uintptr_t)m.ant_n,
                                (long long)(uintptr_t)m.ant_u, (long long)(uintptr_t)m.beam_idx, m.beam_kind,
                                bits(m.gauss_c), m.n_beam, m.n_feed, m.n_ax, m.n_nu, m.n_za, m.n_az, bits(m.dza),
                                bits(m.daz), m.interp};
    const Buf* bufs[] = {&c->R, &c->chan, &c->inst, &c->groups, &c->counts, &c->offsets, &c->le, &c->ln, &c->lu,
                         &c->lidx, &c->lazza, &c->nlive, &c->wa[0], &c->amax[0], &c->sched, &c->u[0], &c->ulo[0],
                         &c->wa[1], &c->amax[1], &c->u[1], &c->ulo[1], &c->wa[2], &c->amax[2], &c->partial,
                         &c->planes, &c->grid, &c->err,
                         &c->lsfix, &c->lseps, &c->aph[0], &c->aph[1], &c->pol_m, &c->red_uidx, &c->red_tl[0],
                         &c->red_tl[1]};
    for (const Buf* b : bufs) k.push_back((long long)(uintptr_t)b->p);
    for (const auto& b : P.batches) {
        k.push_back(b.inst0);
        k.push_back(b.n);
        k.push_back(b.g0);
        k.push_back(b.ng);
    }
    return k;
}

// For the redundant-group output the model's antennas are the cover's order
// (the Z planes are built in that order) for the duration of the call.
struct ModelSwap {
    mv_ctx* c;
    bool on;
    const double *e, *n, *u;
    const int* b;
    ModelSwap(mv_ctx* c_, bool on_) : c(c_), on(on_) {
        Model& m = c->model;
        e = m.ant_e;
        n = m.ant_n;
        u = m.ant_u;
        b = m.beam_idx;
        if (on) {
            m.ant_e = (const double*)c->red_e.p;
            m.ant_n = (const double*)c->red_n.p;
            m.ant_u = (const double*)c->red_u.p;
            m.beam_idx = (const int*)c->red_b.p;
        }
    }
    ~ModelSwap() {
        Model& m = c->model;
        m.ant_e = e;
        m.ant_n = n;
        m.ant_u = u;
        m.beam_idx = b;
    }
};

mv_status run(mv_ctx* c, Plan& P, mv_precision prec, void* V, int V_on_device, cudaStream_t st) {
    c->launches = 0;
    ModelSwap swap(c, P.unique);
    Prepared p;
    mv_status s = prepare(c, P, prec, V, V_on_device, st, p);
    if (s || p.n_inst == 0) return s;
    const HerkCfg h = chosen_cfg(c, p);

    long long L = 0;
    // CUDA graph: the launch sequence is captured once per key (on the
    // context's own stream) and replayed on the caller's stream.  Kernel
    // timing records events around single launches, so it runs uncaptured.
    p.plan = &P;
    if (c->opt.use_graph && !c->profiling && !debug_sync() && !c->use_sur) {
        std::vector<long long> key = graph_key(c, P, p, h);
        if (!c->graph_exec || key != c->graph_key) {
            if (c->graph_exec) {
                cudaGraphExecDestroy(c->graph_exec);
                c->graph_exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            if ((s = cuda_check(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture")))
                return s;
            mv_status se = enqueue_all(c, P, p, h, c->stream, &L);
            cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
            if (se) {
                if (g) cudaGraphDestroy(g);
                return se;
            }
            if ((s = cuda_check(ee, "end capture"))) return s;
            ee = cudaGraphInstantiate(&c->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if ((s = cuda_check(ee, "graph instantiate"))) return s;
            c->graph_key = key;
            c->graph_launches = L;
        }
        if ((s = cuda_check(cudaGraphLaunch(c->graph_exec, st), "graph launch"))) return s;
        L = c->graph_launches;
    } else {
        if ((s = enqueue_all(c, P, p, h, st, &L))) return s;
    }
    c->launches = L;
    c->last_inst_t.clear();
    for (auto& in : P.inst) c->last_inst_t.push_back(in.t);
    if (!V_on_device) {
        if (!p.Vhost &&
            (s = cuda_check(cudaMemcpyAsync(V, p.Vout, p.v_bytes, cudaMemcpyDeviceToHost, st), "copy V to host")))
            return s;
        if ((s = cuda_check(cudaStreamSynchronize(st), "synchronize"))) return s;
        int herr = 0;
        if ((s = cuda_check(cudaMemcpy(&herr, c->err.p, sizeof(int), cudaMemcpyDeviceToHost), "status word")))
            return s;
        if (herr) {
            cudaMemset(c->err.p, 0, sizeof(int));
            return fail(MV_ERR_DEVICE_TIMEOUT, "a device-side wait timed out (code %d); V is invalid", herr);
        }
    }
    return MV_OK;
}

// Autotuner: run the first batch of the call once, then time the HERK of that
// batch under each candidate (tile width, split, flush) with CUDA events and
// keep the fastest for calls of the same shape.  Where the Z build can be
// fused, both schedules are timed per batch -- the fused HERK launch (which
// also builds a batch's Z planes) against the best separate HERK plus the
// batch's own Z-side launches -- and the faster one is kept: the fused
// kernel runs its Z build on a few warps beside the tensor-core roles, which
// pays when the Z build is light (channels stepped within a group) and not
// when every instance needs its own phase evaluation.
mv_status autotune(mv_ctx* c, Plan& P, mv_precision prec, cudaStream_t st, mv_tuning* out) {
    if (prec == MV_PREC_FP32) return fail(MV_ERR_ARG, "the autotuner tunes the tensor-core HERK");
    if (c->use_sur) return fail(MV_ERR_STATE, "autotune with the gridded beam (mv_set_beam_surrogate(ctx, 0))");
    c->tuned.valid = false;
    Prepared p;
    mv_status s;
    if ((s = ensure(c, c->vdev, sizeof(float2)))) return s;
    // V for the trial runs: the context's staging buffer
    if ((s = prepare(c, P, prec, c->vdev.p, 0, st, p))) return s;
    if (p.n_inst == 0) return MV_OK;
    const Plan::Batch b0 = P.batches[0];
    std::vector<HerkCfg> cands;
    const long long est_kb = std::max(1ll, ((long long)c->model.n_ax * c->model.n_src / 2 + 63) / 64);
    // fused trials carry the Z build of the first batch into the second
    // workspace set; separate trials run the HERK alone
    std::vector<bool> fused_trial;
    for (int fz = p.fuse ? 1 : 0; fz >= 0; --fz)
        for (int bn : {128, 256})
            for (int split : {1, 2, 4, 8, 16, 32, 64})
                for (int flush : {4, 8, 16}) {
                    if (split > 1 && est_kb / split < 8) continue;
                    HerkCfg h;
                    h.bn = bn;
                    h.split = split;
                    h.flush = flush;
                    cands.push_back(h);
                    fused_trial.push_back(fz == 1);
                }
    size_t need = 0;
    for (auto& h : cands)
        need = std::max(need, sizeof(float) * 128 * h.bn * (size_t)herk_tc_units(p.rows, p.max_slots, h.split, h.bn));
    if ((s = ensure(c, c->partial, need))) return s;
    long long L = 0;
    const Model& m = c->model;
    cudaError_t e = launch_cull(m, (const double*)c->R.p, p.n_times, p.lt, (int*)c->counts.p, (int*)c->offsets.p,
                                p.bpt, st, &L);
    if ((s = cuda_check(e, "cull"))) return s;
    if (m.beam_kind == 2) {
        e = launch_beam_planes(m, (const float2*)c->grid.p, (const Chan*)c->chan.p, p.n_chan, (float2*)c->planes.p,
                               st, &L);
        if ((s = cuda_check(e, "beam planes"))) return s;
    }
    if ((s = enqueue_zside(c, p, b0, 0, st, &L))) return s;
    ZJob zj{};
    if (p.fuse) {
        if ((s = enqueue_wa(c, p, b0, 1, st, &L))) return s;
        if ((s = enqueue_ant_phase(c, p, b0, 1, st, &L))) return s;
        zj = make_zjob(c, p, b0, 1);
    }
    cudaEvent_t e0 = ev_get(c), e1 = ev_get(c);
    const int reps = 2;
    // the separate schedule's Z side of one batch (beam, phase table, Z build)
    double zside_ms = 0;
    if (p.fuse) {
        if ((s = enqueue_zside(c, p, b0, 1, st, &L))) return s;  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
            if ((s = enqueue_zside(c, p, b0, 1, st, &L))) return s;
        cudaEventRecord(e1, st);
        if ((s = cuda_check(cudaEventSynchronize(e1), "trial timing"))) return s;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        zside_ms = ms / reps;
    }
    HerkCfg best;
    bool best_fused = false;
    double best_ms = 1e300;
    for (size_t i = 0; i < cands.size(); ++i) {
        const HerkCfg& h = cands[i];
        const ZJob* zp = fused_trial[i] ? &zj : nullptr;
        if ((s = cuda_check(enqueue_herk(c, p, b0, h, 0, st, &L, zp), "trial HERK"))) return s;  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
            if ((s = cuda_check(enqueue_herk(c, p, b0, h, 0, st, &L, zp), "trial HERK"))) return s;
        cudaEventRecord(e1, st);
        if ((s = cuda_check(cudaEventSynchronize(e1), "trial timing"))) return s;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per_batch = ms / reps + (p.fuse && !fused_trial[i] ? zside_ms : 0.0);
        if (per_batch < best_ms) {
            best_ms = per_batch;
            best = h;
            best_fused = fused_trial[i];
        }
    }
    c->pool.push_back(e0);
    c->pool.push_back(e1);
    if ((s = mv_check_device_status(c, st))) return s;
    c->tuned.valid = true;
    c->tuned.rows = p.rows;
    c->tuned.slots = p.max_slots;
    c->tuned.zprec = p.zprec;
    c->tuned.cfg = best;
    c->tuned.fuse = best_fused;
    c->tuned.ms = best_ms;
    if (out) {
        out->tile_n = best.bn;
        out->split = best.split;
        out->flush_kblocks = best.flush;
        out->herk_ms = best_ms;
        out->candidates = (int)cands.size();
        out->fused = best_fused ? 1 : 0;
    }
    return MV_OK;
}

}  // namespace

extern "C" {

void mv_default_options(mv_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->interp = MV_INTERP_CUBIC;
    opt->use_graph = 1;
    opt->fuse_zbuild = 1;
}

const char* mv_last_error(void) { return g_err.c_str(); }

mv_status mv_create(mv_ctx** out, int device, const mv_options* opt) {
    g_err.clear();
    if (!out) return fail(MV_ERR_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return fail(MV_ERR_ARG, "no CUDA device %d", device);
    }
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, device) != cudaSuccess) return fail(MV_ERR_CUDA, "device properties");
    if (!(pr.major == 10 && pr.minor == 3))
        return fail(MV_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a", device, pr.major,
                    pr.minor);
    DeviceGuard g(device);
    mv_ctx* c = new mv_ctx();
    c->device = device;
    c->n_sms = pr.multiProcessorCount;
    if (herk_tc_init() != cudaSuccess || mlp_tc_init() != cudaSuccess || gemm_tc_init() != cudaSuccess ||
        mlp_chain_init() != cudaSuccess || wgrad_tc_init() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(MV_ERR_CUDA, "kernel attribute set-up failed");
    }
    mv_default_options(&c->opt);
    if (opt) c->opt = *opt;
    if (c->opt.interp != MV_INTERP_CUBIC && c->opt.interp != MV_INTERP_BILINEAR) {
        delete c;
        return fail(MV_ERR_ARG, "unknown interpolation %d", c->opt.interp);
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->zstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_vdone, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_cdone, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_prep, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_zdone[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_zdone[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_hdone[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_hdone[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        mv_destroy(c);
        return fail(MV_ERR_CUDA, "stream or event creation failed");
    }
    mv_status s = ensure(c, c->err, sizeof(int));
    if (s == MV_OK) s = cuda_check(cudaMemset(c->err.p, 0, sizeof(int)), "status word");
    if (s) {
        mv_destroy(c);
        return s;
    }
    *out = c;
    return MV_OK;
}

void mv_destroy(mv_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    Buf* all[] = {&c->xeq, &c->sqrt_flux, &c->half_alpha, &c->ant_e, &c->ant_n, &c->ant_u, &c->bidx, &c->grid,
                  &c->R, &c->counts, &c->offsets, &c->le, &c->ln, &c->lu, &c->lidx, &c->lazza, &c->nlive,
                  &c->chan, &c->inst, &c->groups, &c->planes, &c->wa[0], &c->amax[0], &c->u[0], &c->ulo[0],
                  &c->wa[1], &c->amax[1], &c->u[1], &c->ulo[1], &c->wa[2], &c->amax[2], &c->vdev, &c->err,
                  &c->partial, &c->sched, &c->lsfix, &c->lseps, &c->aph[0], &c->aph[1], &c->pol_m};
    for (Buf* b : all) buf_free(c, *b);
    surrogate_destroy(c->sur);
    harvest(c);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (cudaEvent_t e : {c->ev_prep, c->ev_zdone[0], c->ev_zdone[1], c->ev_hdone[0], c->ev_hdone[1], c->ev_vdone,
                          c->ev_cdone})
        if (e) cudaEventDestroy(e);
    if (c->zstream) cudaStreamDestroy(c->zstream);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

mv_status mv_init_sky(mv_ctx* c, int64_t n_src, const double* ra, const double* dec, const double* flux_ref,
                      const double* spec_idx, double nu_ref) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_src < 1 || n_src > (int64_t)1 << 30) return fail(MV_ERR_ARG, "n_src %lld out of range", (long long)n_src);
    if (!ra || !dec || !flux_ref) return fail(MV_ERR_ARG, "ra, dec and flux_ref are required");
    if (!(std::isfinite(nu_ref) && nu_ref > 0)) return fail(MV_ERR_ARG, "nu_ref must be positive and finite");
    if (!finite_all(ra, n_src) || !finite_all(dec, n_src)) return fail(MV_ERR_ARG, "ra/dec not finite");
    const int64_t bad_flux =
        first_bad(n_src, [flux_ref](int64_t i) { return std::isfinite(flux_ref[i]) && flux_ref[i] >= 0; });
    if (bad_flux < n_src) return fail(MV_ERR_ARG, "flux_ref[%lld] must be finite and >= 0", (long long)bad_flux);
    if (spec_idx && !finite_all(spec_idx, n_src)) return fail(MV_ERR_ARG, "spec_idx not finite");
    DeviceGuard g(c->device);
    // eq. "xeq": X_eq = (cos ra cos dec, sin ra cos dec, sin dec), SoA
    std::vector<double> xeq(3 * (size_t)n_src);
    std::vector<float> sf(n_src), ha(n_src);
    parallel_for(n_src, [&](int64_t b, int64_t e, int) {
        for (int64_t s = b; s < e; ++s) {
            const double cd = std::cos(dec[s]);
            xeq[s] = std::cos(ra[s]) * cd;
            xeq[n_src + s] = std::sin(ra[s]) * cd;
            xeq[2 * n_src + s] = std::sin(dec[s]);
            sf[s] = (float)std::sqrt(flux_ref[s]);
            ha[s] = spec_idx ? (float)(0.5 * spec_idx[s]) : 0.f;
        }
    });
    mv_status s;
    if ((s = upload(c, c->xeq, xeq.data(), xeq.size() * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->sqrt_flux, sf.data(), sf.size() * sizeof(float), c->stream))) return s;
    if ((s = upload(c, c->half_alpha, ha.data(), ha.size() * sizeof(float), c->stream))) return s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "init_sky"))) return s;
    c->model.n_src = n_src;
    c->model.xeq = (const double*)c->xeq.p;
    c->model.sqrt_flux = (const float*)c->sqrt_flux.p;
    c->model.half_alpha = (const float*)c->half_alpha.p;
    c->model.pol_m = nullptr;
    c->h_flux.assign(flux_ref, flux_ref + n_src);
    c->nu_ref = nu_ref;
    c->have_sky = true;
    return MV_OK;
}

mv_status mv_set_sky_polarisation(mv_ctx* c, int64_t n_src, const double* q, const double* u, const double* v) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (!c->have_sky) return fail(MV_ERR_STATE, "call mv_init_sky first");
    if (!q && !u && !v) {
        c->model.pol_m = nullptr;
            return MV_OK;
    }
    if (!q || !u || !v) return fail(MV_ERR_ARG, "stokes_q, stokes_u and stokes_v go together");
    if (n_src != c->model.n_src) return fail(MV_ERR_ARG, "n_src %lld != the sky's %lld", (long long)n_src,
                                             (long long)c->model.n_src);
    DeviceGuard g(c->device);
    mv_status s;
    const std::vector<double>& fl = c->h_flux;
    // C = [[I + Q, U + iV], [U - iV, I - Q]] = M M^dagger with M lower triangular
    std::vector<float4> M(n_src);
    for (int64_t i = 0; i < n_src; ++i) {
        const double I = fl[i], Q = q[i], U = u[i], V = v[i];
        if (!(std::isfinite(Q) && std::isfinite(U) && std::isfinite(V)))
            return fail(MV_ERR_ARG, "Stokes of source %lld not finite", (long long)i);
        if (Q * Q + U * U + V * V > I * I * (1.0 + 1e-6))
            return fail(MV_ERR_ARG, "source %lld: Q^2 + U^2 + V^2 > I^2", (long long)i);
        const double a = I + Q;
        const double m00 = a > 0.0 ? std::sqrt(a) : 0.0;
        const double m10r = m00 > 0.0 ? U / m00 : 0.0, m10i = m00 > 0.0 ? -V / m00 : 0.0;
        const double d = I - Q - (m10r * m10r + m10i * m10i);
        const double m11 = d > 0.0 ? std::sqrt(d) : 0.0;
        M[i] = make_float4((float)m00, (float)m10r, (float)m10i, (float)m11);
    }
    if ((s = upload(c, c->pol_m, M.data(), M.size() * sizeof(float4), c->stream))) return s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "set_sky_polarisation"))) return s;
    c->model.pol_m = (const float4*)c->pol_m.p;
    return MV_OK;
}

mv_status mv_set_beam_gaussian(mv_ctx* c, double fwhm) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (!(std::isfinite(fwhm) && fwhm > 0)) return fail(MV_ERR_ARG, "fwhm must be positive and finite");
    c->model.beam_kind = 1;
    c->model.gauss_c = (float)(4.0 * std::log(2.0) / (fwhm * fwhm));
    c->model.n_beam = c->model.n_feed = c->model.n_ax = 1;
    c->have_beam = true;
    if (c->have_red && c->red_nf != c->model.n_feed) c->have_red = false;  // the plan's rows per antenna changed
    return MV_OK;
}

mv_status mv_set_beam_grid(mv_ctx* c, int n_beam, int n_feed, int n_ax, int n_nu, int n_za, int n_az,
                           const float* values, double nu0, double dnu, double dza, double daz) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_beam < 1 || (n_feed != 1 && n_feed != 2) || (n_ax != 1 && n_ax != 2))
        return fail(MV_ERR_ARG, "n_beam >= 1, n_feed and n_ax in {1, 2}");
    if (n_nu < 4 || n_za < 3 || n_az < 4 || (n_az & 1))
        return fail(MV_ERR_ARG, "grid needs n_nu >= 4, n_za >= 3 and an even n_az >= 4");
    if (!(std::isfinite(nu0) && std::isfinite(dnu) && dnu > 0 && std::isfinite(dza) && dza > 0 &&
          std::isfinite(daz) && daz > 0))
        return fail(MV_ERR_ARG, "grid spacings must be positive and finite");
    if (std::fabs(n_az * daz - 2 * kPi) > 1e-9 * 2 * kPi) return fail(MV_ERR_ARG, "n_az * daz must equal 2 pi");
    if (!values) return fail(MV_ERR_ARG, "values is NULL");
    const size_t n = (size_t)n_beam * n_feed * n_ax * n_nu * n_za * n_az;
    const int64_t bad = first_bad((int64_t)(2 * n), [values](int64_t i) { return std::isfinite(values[i]); });
    if (bad < (int64_t)(2 * n)) return fail(MV_ERR_ARG, "beam value %zu not finite", (size_t)bad / 2);
    DeviceGuard g(c->device);
    mv_status s;
    if ((s = upload(c, c->grid, values, n * sizeof(float2), c->stream))) return s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "set_beam_grid"))) return s;
    Model& m = c->model;
    m.beam_kind = 2;
    m.n_beam = n_beam;
    m.n_feed = n_feed;
    m.n_ax = n_ax;
    m.n_nu = n_nu;
    m.n_za = n_za;
    m.n_az = n_az;
    m.dza = (float)dza;
    m.daz = (float)daz;
    m.interp = c->opt.interp;
    c->grid_nu0 = nu0;
    c->grid_dnu = dnu;
    c->have_beam = true;
    if (c->have_red && c->red_nf != c->model.n_feed) c->have_red = false;  // the plan's rows per antenna changed
    return MV_OK;
}

mv_status mv_set_antennas(mv_ctx* c, int n_ant, const double* enu, const int32_t* beam_idx, double lat) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_ant < 1 || n_ant > 16384) return fail(MV_ERR_ARG, "n_ant %d out of range", n_ant);
    if (!enu || !finite_all(enu, 3 * (int64_t)n_ant)) return fail(MV_ERR_ARG, "enu missing or not finite");
    if (!std::isfinite(lat) || std::fabs(lat) > kPi / 2) return fail(MV_ERR_ARG, "latitude out of range");
    std::vector<double> e(n_ant), no(n_ant), u(n_ant);
    std::vector<int> b(n_ant, 0);
    for (int a = 0; a < n_ant; ++a) {
        e[a] = enu[3 * a];
        no[a] = enu[3 * a + 1];
        u[a] = enu[3 * a + 2];
        if (beam_idx) {
            if (beam_idx[a] < 0) return fail(MV_ERR_ARG, "beam_idx[%d] < 0", a);
            b[a] = beam_idx[a];
        }
    }
    DeviceGuard g(c->device);
    mv_status s;
    if ((s = upload(c, c->ant_e, e.data(), n_ant * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->ant_n, no.data(), n_ant * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->ant_u, u.data(), n_ant * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->bidx, b.data(), n_ant * sizeof(int), c->stream))) return s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "set_antennas"))) return s;
    Model& m = c->model;
    m.n_ant = n_ant;
    m.ant_e = (const double*)c->ant_e.p;
    m.ant_n = (const double*)c->ant_n.p;
    m.ant_u = (const double*)c->ant_u.p;
    m.beam_idx = (const int*)c->bidx.p;
    c->h_bidx = b;
    c->h_enu.assign(enu, enu + 3 * (size_t)n_ant);
    c->lat = lat;
    c->have_ant = true;
    c->have_red = false;  // a redundancy plan belongs to the antennas it was made for
    return MV_OK;
}

mv_status mv_set_redundancy(mv_ctx* c, double tol_m, int64_t* n_unique) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    c->have_red = false;
    if (tol_m <= 0) return MV_OK;  // off
    if (!c->have_ant || !c->have_beam) return fail(MV_ERR_STATE, "set_antennas and a beam first");
    const Model& m = c->model;
    const int n = m.n_ant, nf = m.n_feed;
    RedPlan& r = c->red;
    const char* why = nullptr;
    if (!plan_redundancy(n, c->h_enu.data(), c->h_bidx.data(), tol_m, nf, 128, r, &why))
        return fail(MV_ERR_ARG, "%s", why);
    // antennas in the cover's order
    std::vector<double> e(n), no(n), u(n);
    std::vector<int> b(n);
    for (int a = 0; a < n; ++a) {
        const int q = r.perm[a];
        e[q] = c->h_enu[3 * a];
        no[q] = c->h_enu[3 * a + 1];
        u[q] = c->h_enu[3 * a + 2];
        b[q] = c->h_bidx[a];
    }
    // group lookup: the entry of V (cover's order) that computes each
    // representative, and whether it is the representative's conjugate
    std::vector<int> uidx((size_t)n * n, -1);
    for (size_t g = 0; g < r.rep_a.size(); ++g) {
        const int a = r.rep_a[g], bb = r.rep_b[g];
        int row, col, cj;
        if (r.kind == 1) { row = r.perm[a]; col = r.perm[bb]; cj = 0; }
        else { row = r.perm[bb]; col = r.perm[a]; cj = 1; }  // kind 2, or the lower triangle
        uidx[(size_t)row * n + col] = 2 * (int)g + cj;
    }
    // tiles of the blocks (rows of U: 2 n_feed per antenna), for 128- and
    // 256-column tiles; at 128 columns every tile is full width
    std::vector<TileDesc> tl[2];
    if (r.kind != 0)
        for (int w = 0; w < 2; ++w) {
            const int BN = w ? 256 : 128;
            for (const RedBlock& k : r.blocks) {
                const int R0 = 2 * nf * k.r0, R1 = 2 * nf * k.r1, C0 = 2 * nf * k.c0, C1 = 2 * nf * k.c1;
                for (int rr = R0; rr < R1; rr += 128)
                    for (int cc = C0; cc < C1; cc += BN) {
                        const int ncol = BN == 128 ? 128 : std::min(256, (C1 - cc + 15) / 16 * 16);
                        tl[w].push_back(TileDesc{rr, cc, ncol, R1, C1, 0, 0, 0});
                    }
            }
        }
    DeviceGuard g(c->device);
    mv_status s;
    if ((s = upload(c, c->red_e, e.data(), n * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->red_n, no.data(), n * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->red_u, u.data(), n * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->red_b, b.data(), n * sizeof(int), c->stream))) return s;
    if ((s = upload(c, c->red_uidx, uidx.data(), uidx.size() * sizeof(int), c->stream))) return s;
    for (int w = 0; w < 2; ++w) {
        c->red_ntl[w] = (int)tl[w].size();
        if (!tl[w].empty() &&
            (s = upload(c, c->red_tl[w], tl[w].data(), tl[w].size() * sizeof(TileDesc), c->stream)))
            return s;
    }
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "set_redundancy"))) return s;
    c->have_red = true;
    c->red_nf = nf;
    if (n_unique) *n_unique = (int64_t)r.rep_a.size();
    return MV_OK;
}

mv_status mv_simulate_unique(mv_ctx* c, int n_t, const double* lst, int n_nu, const double* nu, mv_precision prec,
                             void* V, int V_on_device, void* stream) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_t < 0 || n_nu < 0 || (n_t > 0 && !lst) || (n_nu > 0 && !nu)) return fail(MV_ERR_ARG, "bad time/frequency lists");
    if (!c->have_red) return fail(MV_ERR_STATE, "no redundancy plan (mv_set_redundancy)");
    DeviceGuard g(c->device);
    Plan P;
    plan_grid(c, n_t, lst, n_nu, nu, P);
    P.unique = true;
    const long long per = (long long)c->red.rep_a.size() * c->model.n_feed * c->model.n_feed;
    for (size_t i = 0; i < P.inst.size(); ++i) P.inst[i].v_off = (long long)i * per;
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return run(c, P, prec, V, V_on_device, st);
}

mv_status mv_redundancy_plan(int n_ant, const double* enu, const int32_t* beam_idx, double tol_m, int n_feed,
                             int tile_n, int64_t* n_unique, int32_t* rep_a, int32_t* rep_b, int32_t* group_of,
                             int8_t* conj_of, int32_t* perm, int32_t* kind, int32_t* n_blocks, int32_t* blocks,
                             int64_t* tiles) {
    g_err.clear();
    if (n_ant < 1 || n_ant > 16384) return fail(MV_ERR_ARG, "n_ant %d out of range", n_ant);
    if (!enu || !finite_all(enu, 3 * (int64_t)n_ant)) return fail(MV_ERR_ARG, "enu missing or not finite");
    if (beam_idx)
        for (int a = 0; a < n_ant; ++a)
            if (beam_idx[a] < 0) return fail(MV_ERR_ARG, "beam_idx[%d] < 0", a);
    RedPlan p;
    const char* why = nullptr;
    if (!plan_redundancy(n_ant, enu, beam_idx, tol_m, n_feed, tile_n, p, &why)) return fail(MV_ERR_ARG, "%s", why);
    const long long n_bl = (long long)n_ant * (n_ant + 1) / 2;
    if (n_unique) *n_unique = (int64_t)p.rep_a.size();
    if (rep_a) std::memcpy(rep_a, p.rep_a.data(), sizeof(int32_t) * p.rep_a.size());
    if (rep_b) std::memcpy(rep_b, p.rep_b.data(), sizeof(int32_t) * p.rep_b.size());
    if (group_of) std::memcpy(group_of, p.group_of.data(), sizeof(int32_t) * n_bl);
    if (conj_of) std::memcpy(conj_of, p.conj_of.data(), (size_t)n_bl);
    if (perm) std::memcpy(perm, p.perm.data(), sizeof(int32_t) * n_ant);
    if (kind) *kind = p.kind;
    if (n_blocks) *n_blocks = (int32_t)p.blocks.size();
    if (blocks)
        for (size_t i = 0; i < p.blocks.size(); ++i) {
            blocks[4 * i] = p.blocks[i].r0;
            blocks[4 * i + 1] = p.blocks[i].r1;
            blocks[4 * i + 2] = p.blocks[i].c0;
            blocks[4 * i + 3] = p.blocks[i].c1;
        }
    if (tiles) {
        tiles[0] = p.tiles;
        tiles[1] = p.tiles_full;
    }
    return MV_OK;
}

mv_status mv_simulate(mv_ctx* c, int n_t, const double* lst, int n_nu, const double* nu, mv_precision prec,
                      void* V, int V_on_device, void* stream) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_t < 0 || n_nu < 0 || (n_t > 0 && !lst) || (n_nu > 0 && !nu)) return fail(MV_ERR_ARG, "bad time/frequency lists");
    DeviceGuard g(c->device);
    Plan P;
    plan_grid(c, n_t, lst, n_nu, nu, P);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return run(c, P, prec, V, V_on_device, st);
}

mv_status mv_simulate_pairs(mv_ctx* c, int n_pairs, const double* lst, const double* nu, mv_precision prec, void* V,
                            int V_on_device, void* stream) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_pairs < 0 || (n_pairs > 0 && (!lst || !nu))) return fail(MV_ERR_ARG, "bad pair lists");
    DeviceGuard g(c->device);
    Plan P;
    plan_pairs(c, n_pairs, lst, nu, P);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return run(c, P, prec, V, V_on_device, st);
}

mv_status mv_autotune(mv_ctx* c, int n_t, const double* lst, int n_nu, const double* nu, mv_precision prec,
                      int pairs, mv_tuning* out) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_t < 1 || n_nu < 1 || !lst || !nu || (pairs && n_t != n_nu))
        return fail(MV_ERR_ARG, "bad time/frequency lists");
    DeviceGuard g(c->device);
    Plan P;
    if (pairs) plan_pairs(c, n_t, lst, nu, P);
    else plan_grid(c, n_t, lst, n_nu, nu, P);
    return autotune(c, P, prec, c->stream, out);
}

mv_status mv_check_device_status(mv_ctx* c, void* stream) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    DeviceGuard g(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    mv_status s;
    if ((s = cuda_check(cudaStreamSynchronize(st), "synchronize"))) return s;
    int herr = 0;
    if ((s = cuda_check(cudaMemcpy(&herr, c->err.p, sizeof(int), cudaMemcpyDeviceToHost), "status word"))) return s;
    if (herr) {
        cudaMemset(c->err.p, 0, sizeof(int));
        return fail(MV_ERR_DEVICE_TIMEOUT, "a device-side wait timed out (code %d)", herr);
    }
    return MV_OK;
}

mv_status mv_selftest_wait_timeout(mv_ctx* c, double limit_s) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (!(limit_s > 0) || limit_s > 10) return fail(MV_ERR_ARG, "limit_s must be in (0, 10]");
    DeviceGuard g(c->device);
    mv_status s;
    if ((s = cuda_check(launch_wait_probe((int*)c->err.p, limit_s, c->stream), "wait probe"))) return s;
    return mv_check_device_status(c, nullptr);
}

mv_status mv_last_live_counts(mv_ctx* c, int n, int64_t* out) {
    g_err.clear();
    if (!c || !out) return fail(MV_ERR_ARG, "NULL argument");
    if (n != (int)c->last_inst_t.size()) return fail(MV_ERR_ARG, "n must equal the last call's instance count");
    if (n == 0) return MV_OK;
    DeviceGuard g(c->device);
    int n_times = 0;
    for (int t : c->last_inst_t) n_times = std::max(n_times, t + 1);
    std::vector<int> h(n_times);
    mv_status s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "synchronize"))) return s;
    if ((s = cuda_check(cudaDeviceSynchronize(), "synchronize"))) return s;
    if ((s = cuda_check(cudaMemcpy(h.data(), c->nlive.p, n_times * sizeof(int), cudaMemcpyDeviceToHost), "n_live")))
        return s;
    for (int i = 0; i < n; ++i) out[i] = h[c->last_inst_t[i]];
    return MV_OK;
}

int64_t mv_last_launch_count(mv_ctx* c) { return c ? c->launches : -1; }

mv_status mv_profile_enable(mv_ctx* c, int enable) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    DeviceGuard g(c->device);
    harvest(c);
    for (int k = 0; k < MV_KERNEL_KINDS; ++k) {
        c->prof_launches[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    c->profiling = enable != 0;
    return MV_OK;
}

mv_status mv_profile_read(mv_ctx* c, int kind, int64_t* launches, double* total_ms) {
    g_err.clear();
    if (!c || !launches || !total_ms) return fail(MV_ERR_ARG, "NULL argument");
    if (kind < 0 || kind >= MV_KERNEL_KINDS) return fail(MV_ERR_ARG, "unknown kernel kind %d", kind);
    DeviceGuard g(c->device);
    harvest(c);
    *launches = c->prof_launches[kind];
    *total_ms = c->prof_ms[kind];
    return MV_OK;
}

void mv_default_mlp_config(mv_mlp_config* cfg) {
    if (!cfg) return;
    cfg->n_freq = 64;
    cfg->emb_dim = 16;
    cfg->width = 256;
    cfg->depth = 4;
    cfg->sigma_az = 2.f;
    cfg->sigma_za = 3.f;
    cfg->sigma_nu = 1.f;
    cfg->seed = 20231213ull;
}

mv_status mv_surrogate_create(mv_ctx* c, const mv_mlp_config* cfg) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (c->model.beam_kind != 2) return fail(MV_ERR_STATE, "the surrogate learns a gridded beam: set one first");
    mv_mlp_config k;
    mv_default_mlp_config(&k);
    if (cfg) k = *cfg;
    if (k.n_freq < 1 || k.emb_dim < 1 || 2 * k.n_freq + k.emb_dim > 240 || k.width < 64 || k.width > 256 ||
        k.width % 16 || k.depth < 1 || k.depth > 16)
        return fail(MV_ERR_ARG, "MLP configuration out of range (width a multiple of 16 in [64, 256], 2 n_freq + "
                                "emb_dim <= 240, depth 1-16)");
    DeviceGuard g(c->device);
    const Model& m = c->model;
    const double nu_lo = c->grid_nu0, nu_hi = c->grid_nu0 + (m.n_nu - 1) * c->grid_dnu;
    cudaError_t e = cudaSuccess;
    Surrogate* S = surrogate_create(k.n_freq, k.emb_dim, k.width, k.depth, 2 * m.n_feed * m.n_ax, m.n_beam,
                                    k.sigma_az, k.sigma_za, k.sigma_nu, k.seed, 0.5 * (nu_lo + nu_hi),
                                    0.5 * (nu_hi - nu_lo), &e);
    if (!S) return fail(MV_ERR_OOM, "surrogate allocation failed: %s", cudaGetErrorString(e));
    surrogate_destroy(c->sur);
    c->sur = S;
    c->sur_cfg = k;
    return MV_OK;
}

mv_status mv_surrogate_train(mv_ctx* c, int steps, int batch, float lr0, float lr1, uint64_t seed,
                             double* loss_first, double* loss_last) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (!c->sur) return fail(MV_ERR_STATE, "no surrogate: call mv_surrogate_create");
    if (steps < 1 || batch < 8 || batch % 8 || batch > (1 << 24) || !(lr0 > 0) || !(lr1 >= 0))
        return fail(MV_ERR_ARG, "steps >= 1, batch a multiple of 8, lr0 > 0, lr1 >= 0");
    DeviceGuard g(c->device);
    double l0 = 0, l1 = 0;
    long long L = 0;
    cudaError_t e = surrogate_train(c->sur, c->model, (const float2*)c->grid.p, c->grid_nu0, c->grid_dnu, steps, batch,
                                    lr0, lr1, seed, c->stream, &l0, &l1, &L);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(MV_ERR_CUDA, "surrogate training: %s", cudaGetErrorString(e));
    if (loss_first) *loss_first = l0;
    if (loss_last) *loss_last = l1;
    c->launches = L;
    return MV_OK;
}

mv_status mv_surrogate_params(mv_ctx* c, int64_t* n_params, float* host, float* fourier, int64_t* layout) {
    g_err.clear();
    if (!c || !n_params) return fail(MV_ERR_ARG, "NULL argument");
    if (!c->sur) return fail(MV_ERR_STATE, "no surrogate");
    DeviceGuard g(c->device);
    *n_params = surrogate_param_count(c->sur);
    if (host) {
        cudaError_t e = surrogate_get_params(c->sur, host);
        if (e != cudaSuccess) return fail(MV_ERR_CUDA, "parameter copy: %s", cudaGetErrorString(e));
    }
    if (fourier) surrogate_fourier(c->sur, fourier);
    if (layout) {
        const int D = c->sur_cfg.depth;
        std::vector<long long> ow(D + 1), ob(D + 1);
        long long oe = 0;
        int d0p = 0;
        surrogate_layout(c->sur, ow.data(), ob.data(), &oe, &d0p);
        for (int l = 0; l <= D; ++l) {
            layout[2 * l] = ow[l];
            layout[2 * l + 1] = ob[l];
        }
        layout[2 * (D + 1)] = oe;
        layout[2 * (D + 1) + 1] = d0p;
    }
    return MV_OK;
}

mv_status mv_surrogate_set_params(mv_ctx* c, const float* host) {
    g_err.clear();
    if (!c || !host) return fail(MV_ERR_ARG, "NULL argument");
    if (!c->sur) return fail(MV_ERR_STATE, "no surrogate");
    DeviceGuard g(c->device);
    cudaError_t e = surrogate_set_params(c->sur, host);
    if (e != cudaSuccess) return fail(MV_ERR_CUDA, "parameter copy: %s", cudaGetErrorString(e));
    return MV_OK;
}

namespace {
mv_status points(mv_ctx* c, int n, const int32_t* beam, const double* az, const double* za, const double* nu,
                 std::vector<float>& faz, std::vector<float>& fza, std::vector<float>& fnu) {
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (!c->sur) return fail(MV_ERR_STATE, "no surrogate");
    if (n < 1 || !beam || !az || !za || !nu) return fail(MV_ERR_ARG, "bad point arrays");
    faz.resize(n);
    fza.resize(n);
    fnu.resize(n);
    for (int i = 0; i < n; ++i) {
        if (beam[i] < 0 || beam[i] >= c->model.n_beam) return fail(MV_ERR_ARG, "beam index %d out of range", beam[i]);
        if (!std::isfinite(az[i]) || !std::isfinite(za[i]) || !std::isfinite(nu[i]))
            return fail(MV_ERR_ARG, "point %d not finite", i);
        faz[i] = (float)az[i];
        fza[i] = (float)za[i];
        fnu[i] = (float)nu[i];
    }
    return MV_OK;
}
}  // namespace

mv_status mv_surrogate_eval(mv_ctx* c, int n, const int32_t* beam, const double* az, const double* za,
                            const double* nu, float* out) {
    g_err.clear();
    std::vector<float> faz, fza, fnu;
    mv_status s = points(c, n, beam, az, za, nu, faz, fza, fnu);
    if (s) return s;
    if (!out) return fail(MV_ERR_ARG, "out is NULL");
    DeviceGuard g(c->device);
    cudaError_t e = surrogate_eval(c->sur, n, beam, faz.data(), fza.data(), fnu.data(), out, c->stream);
    if (e != cudaSuccess) return fail(MV_ERR_CUDA, "surrogate evaluation: %s", cudaGetErrorString(e));
    return MV_OK;
}

mv_status mv_surrogate_grad(mv_ctx* c, int n, const int32_t* beam, const double* az, const double* za,
                            const double* nu, const float* target, float* grads, double* loss) {
    g_err.clear();
    std::vector<float> faz, fza, fnu;
    mv_status s = points(c, n, beam, az, za, nu, faz, fza, fnu);
    if (s) return s;
    if (n % 8 || !target || !grads || !loss) return fail(MV_ERR_ARG, "n a multiple of 8; target, grads, loss");
    DeviceGuard g(c->device);
    cudaError_t e = surrogate_grad(c->sur, n, beam, faz.data(), fza.data(), fnu.data(), target, grads, loss, c->stream);
    if (e != cudaSuccess) return fail(MV_ERR_CUDA, "surrogate gradient: %s", cudaGetErrorString(e));
    return MV_OK;
}

mv_status mv_surrogate_save(mv_ctx* c, const char* path) {
    g_err.clear();
    if (!c || !path) return fail(MV_ERR_ARG, "NULL argument");
    if (!c->sur) return fail(MV_ERR_STATE, "no surrogate");
    DeviceGuard g(c->device);
    const long long n = surrogate_param_count(c->sur);
    std::vector<float> p(n), B(3 * (size_t)c->sur_cfg.n_freq);
    if (surrogate_get_params(c->sur, p.data()) != cudaSuccess) return fail(MV_ERR_CUDA, "parameter copy");
    surrogate_fourier(c->sur, B.data());
    FILE* f = fopen(path, "wb");
    if (!f) return fail(MV_ERR_ARG, "cannot open %s for writing", path);
    const char magic[8] = {'M', 'V', 'M', 'L', 'P', '0', '0', '1'};
    const int32_t hdr[6] = {c->sur_cfg.n_freq, c->sur_cfg.emb_dim, c->sur_cfg.width, c->sur_cfg.depth,
                            c->model.n_beam, 2 * c->model.n_feed * c->model.n_ax};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(&c->sur_cfg, sizeof(mv_mlp_config), 1, f) == 1 && fwrite(&n, sizeof(n), 1, f) == 1 &&
              fwrite(B.data(), sizeof(float), B.size(), f) == B.size() &&
              fwrite(p.data(), sizeof(float), (size_t)n, f) == (size_t)n;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(MV_ERR_ARG, "write to %s failed", path);
    return MV_OK;
}

mv_status mv_surrogate_load(mv_ctx* c, const char* path) {
    g_err.clear();
    if (!c || !path) return fail(MV_ERR_ARG, "NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(MV_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t hdr[6];
    mv_mlp_config k;
    long long n = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "MVMLP001", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              fread(&k, sizeof(k), 1, f) == 1 && fread(&n, sizeof(n), 1, f) == 1;
    std::vector<float> B, p;
    if (ok) {
        B.resize(3 * (size_t)std::max(0, hdr[0]));
        p.resize((size_t)std::max(0ll, n));
        ok = fread(B.data(), sizeof(float), B.size(), f) == B.size() && fread(p.data(), sizeof(float), p.size(), f) == p.size();
    }
    fclose(f);
    if (!ok) return fail(MV_ERR_ARG, "%s is not a surrogate file", path);
    if (hdr[4] != c->model.n_beam || hdr[5] != 2 * c->model.n_feed * c->model.n_ax)
        return fail(MV_ERR_ARG, "surrogate in %s was made for another beam set", path);
    mv_status s = mv_surrogate_create(c, &k);  // same seed: the same B
    if (s) return s;
    std::vector<float> B2(B.size());
    surrogate_fourier(c->sur, B2.data());
    if (B2 != B || surrogate_param_count(c->sur) != n) return fail(MV_ERR_ARG, "surrogate file layout mismatch");
    return mv_surrogate_set_params(c, p.data());
}

mv_status mv_set_beam_surrogate(mv_ctx* c, int enable) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (enable && !c->sur) return fail(MV_ERR_STATE, "no surrogate");
    c->use_sur = enable != 0;
    return MV_OK;
}

mv_status mv_beam_model_bytes(mv_ctx* c, int64_t* grid_bytes, int64_t* surrogate_bytes) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (grid_bytes) *grid_bytes = c->model.beam_kind == 2 ? (int64_t)(c->grid.bytes + c->planes.bytes) : 0;
    if (surrogate_bytes) *surrogate_bytes = c->sur ? surrogate_eval_bytes(c->sur) : 0;
    return MV_OK;
}

}  // extern "C"
