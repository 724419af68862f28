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
#include <vector>

#include "matvis.h"
#include "common.cuh"

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
    double grid_nu0 = 0, grid_dnu = 0;
    // model buffers
    Buf xeq, sqrt_flux, half_alpha, ant_e, ant_n, ant_u, bidx, grid;
    // workspace
    Buf R, counts, offsets, le, ln, lu, lidx, lazza, nlive, chan, inst, groups, planes, wa, amax, u, ulo, vdev, err;
    long long launches = 0;
    std::vector<int> last_inst_t;
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

bool finite_all(const double* p, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
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
    if (c->opt.max_batch > 0) return c->opt.max_batch;
    const long long budget = 8ll << 30;  // workspace for the Z planes
    long long b = budget / std::max(slot_bytes, 1ll);
    return (int)std::max(1ll, std::min(b, 16ll));
}

mv_status run(mv_ctx* c, Plan& P, mv_precision prec, void* V, int V_on_device, cudaStream_t st) {
    Model& m = c->model;
    if (!c->have_sky || !c->have_ant || !c->have_beam)
        return fail(MV_ERR_STATE, "simulate needs init_sky, set_antennas and a beam first");
    if (prec != MV_PREC_FP32 && prec != MV_PREC_BF16X3 && prec != MV_PREC_FP16X3)
        return fail(MV_ERR_ARG, "unknown precision %d", (int)prec);
    if (!V) return fail(MV_ERR_ARG, "V is NULL");
    if (prec != MV_PREC_FP32 && !herk_tc_available())
        return fail(MV_ERR_UNSUPPORTED, "tensor-map encoding unavailable in this driver");
    for (int b : c->h_bidx)
        if (b >= m.n_beam) return fail(MV_ERR_ARG, "antenna beam index %d >= n_beam %d", b, m.n_beam);
    const int n_times = (int)P.lst.size(), n_chan = (int)P.nu.size();
    const int n_inst = (int)P.inst.size();
    c->launches = 0;
    if (n_inst == 0) return MV_OK;

    // channel table
    std::vector<Chan> chan(n_chan);
    for (int i = 0; i < n_chan; ++i) {
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
    std::vector<double> R(9 * (size_t)n_times);
    const double sl = std::sin(c->lat), cl = std::cos(c->lat);
    for (int t = 0; t < n_times; ++t) {
        if (!std::isfinite(P.lst[t])) return fail(MV_ERR_ARG, "LST %d is not finite", t);
        const double H = -P.lst[t];
        const double sH = std::sin(H), cH = std::cos(H);
        double* r = &R[9 * (size_t)t];
        r[0] = sH;        r[1] = cH;        r[2] = 0.0;
        r[3] = -sl * cH;  r[4] = sl * sH;   r[5] = cl;
        r[6] = cl * cH;   r[7] = -cl * sH;  r[8] = sl;
    }

    // sizes
    const int N = m.n_feed * m.n_ant;
    const int rows = 2 * N;
    const long long pitch = round_up(m.n_src, kKPad);
    const long long k_pitch = round_up((long long)m.n_ax * m.n_src, kKPad);
    const int bpt = (int)((m.n_src + 255) / 256);
    const int ncomp = m.n_beam * m.n_feed * m.n_ax;
    int max_slots = 0;
    for (auto& b : P.batches) max_slots = std::max(max_slots, b.n);

    mv_status s;
    if ((s = upload(c, c->R, R.data(), R.size() * sizeof(double), st))) return s;
    if ((s = upload(c, c->chan, chan.data(), chan.size() * sizeof(Chan), st))) return s;
    if ((s = upload(c, c->inst, P.inst.data(), P.inst.size() * sizeof(Inst), st))) return s;
    if ((s = upload(c, c->groups, P.groups.data(), P.groups.size() * sizeof(ZGroup), st))) return s;
    if ((s = ensure(c, c->counts, sizeof(int) * (size_t)bpt * n_times))) return s;
    if ((s = ensure(c, c->offsets, sizeof(int) * (size_t)bpt * n_times))) return s;
    if ((s = ensure(c, c->le, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->ln, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lu, sizeof(double) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lidx, sizeof(int) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->lazza, sizeof(float2) * (size_t)pitch * n_times))) return s;
    if ((s = ensure(c, c->nlive, sizeof(int) * (size_t)n_times))) return s;
    if ((s = ensure(c, c->wa, sizeof(float2) * (size_t)max_slots * ncomp * pitch))) return s;
    if ((s = ensure(c, c->amax, sizeof(float) * (size_t)max_slots))) return s;
    const size_t plane_elems = (size_t)rows * k_pitch * max_slots;
    if (prec == MV_PREC_FP32) {
        if ((s = ensure(c, c->u, sizeof(float) * plane_elems))) return s;
    } else {
        if ((s = ensure(c, c->u, 2 * plane_elems))) return s;
        if ((s = ensure(c, c->ulo, 2 * plane_elems))) return s;
    }
    if (m.beam_kind == 2 &&
        (s = ensure(c, c->planes, sizeof(float2) * (size_t)n_chan * ncomp * m.n_za * m.n_az)))
        return s;
    float2* Vout = static_cast<float2*>(V);
    const size_t v_bytes = sizeof(float2) * (size_t)n_inst * N * N;
    if (!V_on_device) {
        if ((s = ensure(c, c->vdev, v_bytes))) return s;
        Vout = static_cast<float2*>(c->vdev.p);
    }

    LiveTables lt;
    lt.e = (double*)c->le.p;
    lt.n = (double*)c->ln.p;
    lt.u = (double*)c->lu.p;
    lt.idx = (int*)c->lidx.p;
    lt.azza = (float2*)c->lazza.p;
    lt.n_live = (int*)c->nlive.p;
    lt.pitch = pitch;

    long long L = 0;
    Timed tc0(c, MV_KERNEL_CULL, st);
    cudaError_t e = launch_cull(m, (const double*)c->R.p, n_times, lt, (int*)c->counts.p, (int*)c->offsets.p, bpt,
                                st, &L);
    tc0.end();
    if ((s = launched(e, "cull", st))) return s;
    if (m.beam_kind == 2) {
        Timed tb(c, MV_KERNEL_BEAM, st);
        e = launch_beam_planes(m, (const float2*)c->grid.p, (const Chan*)c->chan.p, n_chan, (float2*)c->planes.p, st,
                               &L);
        tb.end();
        if ((s = launched(e, "beam planes", st))) return s;
    }
    const Inst* d_inst = (const Inst*)c->inst.p;
    const int zprec = prec == MV_PREC_FP32 ? 0 : (prec == MV_PREC_BF16X3 ? 1 : 2);
    for (const auto& b : P.batches) {
        if ((s = cuda_check(cudaMemsetAsync(c->amax.p, 0, sizeof(float) * b.n, st), "amax reset"))) return s;
        Timed tw(c, MV_KERNEL_BEAM, st);
        e = launch_wa(m, (const float2*)c->planes.p, (const Chan*)c->chan.p, d_inst, b.inst0, b.n, lt,
                      (float2*)c->wa.p, pitch, (float*)c->amax.p, st, &L);
        tw.end();
        if ((s = launched(e, "beam evaluation", st))) return s;
        Timed tz(c, MV_KERNEL_ZBUILD, st);
        e = launch_zbuild(m, d_inst, (const Chan*)c->chan.p, (const ZGroup*)c->groups.p, b.g0, b.ng, lt,
                          (const float2*)c->wa.p, pitch, (const float*)c->amax.p, c->u.p, c->ulo.p, zprec, rows,
                          k_pitch, st, &L);
        tz.end();
        if ((s = launched(e, "Z build", st))) return s;
        Timed th(c, MV_KERNEL_HERK, st);
        if (prec == MV_PREC_FP32) {
            e = launch_herk_fp32(d_inst, b.inst0, b.n, lt, m.n_ax, (const float*)c->u.p, rows, k_pitch, Vout, N, 256,
                                 st, &L);
        } else {
            const int flush = c->opt.herk_flush_kblocks > 0 ? c->opt.herk_flush_kblocks : 4;
            e = launch_herk_tc(d_inst, b.inst0, b.n, lt, m.n_ax, (const __nv_bfloat16*)c->u.p,
                               (const __nv_bfloat16*)c->ulo.p, rows, k_pitch, max_slots, zprec == 2 ? 1 : 0,
                               (const float*)c->amax.p, Vout, N, flush, (int*)c->err.p, st, &L);
        }
        th.end();
        if ((s = launched(e, zprec == 0 ? "HERK fp32" : "HERK tc", st))) return s;
    }
    c->launches = L;
    c->last_inst_t.clear();
    for (auto& in : P.inst) c->last_inst_t.push_back(in.t);
    if (!V_on_device) {
        if ((s = cuda_check(cudaMemcpyAsync(V, Vout, v_bytes, cudaMemcpyDeviceToHost, st), "copy V to host")))
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

}  // namespace

extern "C" {

void mv_default_options(mv_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->interp = MV_INTERP_CUBIC;
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
    mv_default_options(&c->opt);
    if (opt) c->opt = *opt;
    if (c->opt.interp != MV_INTERP_CUBIC && c->opt.interp != MV_INTERP_BILINEAR) {
        delete c;
        return fail(MV_ERR_ARG, "unknown interpolation %d", c->opt.interp);
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return fail(MV_ERR_CUDA, "stream creation failed");
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
                  &c->chan, &c->inst, &c->groups, &c->planes, &c->wa, &c->amax, &c->u, &c->ulo, &c->vdev, &c->err};
    for (Buf* b : all) buf_free(c, *b);
    harvest(c);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
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
    for (int64_t i = 0; i < n_src; ++i)
        if (!(std::isfinite(flux_ref[i]) && flux_ref[i] >= 0))
            return fail(MV_ERR_ARG, "flux_ref[%lld] must be finite and >= 0", (long long)i);
    if (spec_idx && !finite_all(spec_idx, n_src)) return fail(MV_ERR_ARG, "spec_idx not finite");
    DeviceGuard g(c->device);
    // eq. "xeq": X_eq = (cos ra cos dec, sin ra cos dec, sin dec), SoA
    std::vector<double> xeq(3 * (size_t)n_src);
    std::vector<float> sf(n_src), ha(n_src);
    for (int64_t s = 0; s < n_src; ++s) {
        const double cd = std::cos(dec[s]);
        xeq[s] = std::cos(ra[s]) * cd;
        xeq[n_src + s] = std::sin(ra[s]) * cd;
        xeq[2 * n_src + s] = std::sin(dec[s]);
        sf[s] = (float)std::sqrt(flux_ref[s]);
        ha[s] = spec_idx ? (float)(0.5 * spec_idx[s]) : 0.f;
    }
    mv_status s;
    if ((s = upload(c, c->xeq, xeq.data(), xeq.size() * sizeof(double), c->stream))) return s;
    if ((s = upload(c, c->sqrt_flux, sf.data(), sf.size() * sizeof(float), c->stream))) return s;
    if ((s = upload(c, c->half_alpha, ha.data(), ha.size() * sizeof(float), c->stream))) return s;
    if ((s = cuda_check(cudaStreamSynchronize(c->stream), "init_sky"))) return s;
    c->model.n_src = n_src;
    c->model.xeq = (const double*)c->xeq.p;
    c->model.sqrt_flux = (const float*)c->sqrt_flux.p;
    c->model.half_alpha = (const float*)c->half_alpha.p;
    c->nu_ref = nu_ref;
    c->have_sky = true;
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
    for (size_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(values[i])) return fail(MV_ERR_ARG, "beam value %zu not finite", i / 2);
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
    c->lat = lat;
    c->have_ant = true;
    return MV_OK;
}

mv_status mv_simulate(mv_ctx* c, int n_t, const double* lst, int n_nu, const double* nu, mv_precision prec,
                      void* V, int V_on_device, void* stream) {
    g_err.clear();
    if (!c) return fail(MV_ERR_ARG, "ctx is NULL");
    if (n_t < 0 || n_nu < 0 || (n_t > 0 && !lst) || (n_nu > 0 && !nu)) return fail(MV_ERR_ARG, "bad time/frequency lists");
    DeviceGuard g(c->device);
    Plan P;
    P.lst.assign(lst, lst + n_t);
    P.nu.assign(nu, nu + n_nu);
    const long long N = (long long)c->model.n_feed * c->model.n_ant;
    for (int t = 0; t < n_t; ++t)
        for (int f = 0; f < n_nu; ++f) P.inst.push_back(Inst{t, f, ((long long)t * n_nu + f) * N * N});
    const long long slot_bytes = 4ll * 2 * N * round_up((long long)c->model.n_ax * std::max<long long>(c->model.n_src, 1), kKPad);
    const int B = auto_batch(c, slot_bytes);
    for (int t = 0; t < n_t; ++t)
        for (int f0 = 0; f0 < n_nu; f0 += B) {
            const int n = std::min(B, n_nu - f0);
            const int i0 = t * n_nu + f0;
            Plan::Batch b{i0, n, (int)P.groups.size(), 1};
            P.groups.push_back(make_group(P, i0, n, 0));
            P.batches.push_back(b);
        }
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
    P.lst.assign(lst, lst + n_pairs);
    P.nu.assign(nu, nu + n_pairs);
    const long long N = (long long)c->model.n_feed * c->model.n_ant;
    for (int i = 0; i < n_pairs; ++i) P.inst.push_back(Inst{i, i, (long long)i * N * N});
    const long long slot_bytes = 4ll * 2 * N * round_up((long long)c->model.n_ax * std::max<long long>(c->model.n_src, 1), kKPad);
    const int B = auto_batch(c, slot_bytes);
    for (int i0 = 0; i0 < n_pairs; i0 += B) {
        const int n = std::min(B, n_pairs - i0);
        Plan::Batch b{i0, n, (int)P.groups.size(), n};
        for (int j = 0; j < n; ++j) P.groups.push_back(make_group(P, i0 + j, 1, j));
        P.batches.push_back(b);
    }
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return run(c, P, prec, V, V_on_device, st);
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

}  // extern "C"
