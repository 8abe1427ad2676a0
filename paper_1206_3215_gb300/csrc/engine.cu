// Stepping drivers: which passes run, in which order, on which buffers.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "engine.h"
#include "plan.h"
#include "tables.h"

using namespace pss;

namespace {
// the device status word pass kernels report a lost tile copy in
int *pass_status(pss_grid *g) { return reinterpret_cast<int *>(g->flags) + FLAG_SLOT_PASS_STATUS; }
}  // namespace

namespace {

template <class Rl> V2<Rl> *B(pss_grid *g, int i) { return static_cast<V2<Rl> *>(g->buf[i]); }
template <class Rl> const V2<Rl> *C(const void *p) { return static_cast<const V2<Rl> *>(p); }
template <class Rl> const TW<Rl> *Tw(const void *p) { return static_cast<const TW<Rl> *>(p); }

cudaMemcpyKind kind_in(int where) { return where == PSS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind kind_out(int where) { return where == PSS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

// Upload a per-axis table of n complex values given by f(m) -> (re, im) in FP64,
// in the twiddle layout of the grid's precision (FP32: hi + lo quadruples).
template <class F> int upload_cplx_table(pss_grid *g, int64_t n, F f, void **dst)
{
    if (g->p.precision == PSS_FP32) {
        std::vector<float> t(4 * n);
        for (int64_t m = 0; m < n; ++m) {
            double re, im;
            f(m, &re, &im);
            hilo_f32(re, im, &t[4 * m]);
        }
        return g->upload(dst, t.data(), t.size() * 4);
    }
    std::vector<double> t(2 * n);
    for (int64_t m = 0; m < n; ++m) f(m, &t[2 * m], &t[2 * m + 1]);
    return g->upload(dst, t.data(), t.size() * 8);
}

int upload_twiddles(pss_grid *g, int64_t n, void **dst)
{
    if (g->p.precision == PSS_FP32) {
        auto t = twiddles_f32(n);
        return g->upload(dst, t.data(), t.size() * 4);
    }
    auto t = twiddles_f64(n);
    return g->upload(dst, t.data(), t.size() * 8);
}

template <class Rl> int upload_real(pss_grid *g, const std::vector<double> &v, void **dst)
{
    std::vector<Rl> r(v.begin(), v.end());
    return g->upload(dst, r.data(), r.size() * sizeof(Rl));
}

}  // namespace

// ----------------------------------------------------------------------------

int pss_grid::init()
{
    nx = p.nx;
    ny = p.ny;
    batch = p.batch;
    npts = nx * ny;
    ntot = npts * batch;
    esz = p.precision == PSS_FP32 ? 8 : 16;
    int rc;
    if ((rc = cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (p.stream) {
        stream = static_cast<cudaStream_t>(p.stream);
    } else {
        if ((rc = cuda(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "stream"))) return rc;
        own_stream = true;
    }
    {
        const char *gr = getenv("PSS_GRAPHS");
        use_graphs = !(gr && gr[0] == '0');
    }
    // work arrays
    nbuf = p.eq == PSS_EQ_NLS ? 3 : p.eq == PSS_EQ_SG ? 5 : 7;
    for (int i = 0; i < nbuf; ++i) {
        if ((rc = alloc(&buf[i], field_bytes()))) return rc;
        if ((rc = cuda(cudaMemset(buf[i], 0, field_bytes()), "memset"))) return rc;
    }
    // tables
    if ((rc = upload_twiddles(this, nx, &twx))) return rc;
    if ((rc = upload_twiddles(this, ny, &twy))) return rc;
    std::vector<double> kx2v(nx), ky2v(ny), kxov(nx), kyov(ny), kpx(nx), kpy(ny);
    for (int64_t m = 0; m < nx; ++m) {
        const double k = wavenumber(m, nx, p.lx);
        kx2v[m] = k * k;
        kxov[m] = (m == nx / 2) ? 0.0 : k;
        kpx[m] = (!p.dealias || 3 * std::llabs(m < nx / 2 ? m : m - nx) < nx) ? 1.0 : 0.0;
    }
    for (int64_t m = 0; m < ny; ++m) {
        const double k = wavenumber(m, ny, p.ly);
        ky2v[m] = k * k;
        kyov[m] = (m == ny / 2) ? 0.0 : k;
        kpy[m] = (!p.dealias || 3 * std::llabs(m < ny / 2 ? m : m - ny) < ny) ? 1.0 : 0.0;
    }
    if ((rc = upload((void **)&kx2d, kx2v.data(), nx * 8))) return rc;
    if ((rc = upload((void **)&ky2d, ky2v.data(), ny * 8))) return rc;
    if (p.precision == PSS_FP32) {
        if ((rc = upload_real<float>(this, kx2v, &kx2)) || (rc = upload_real<float>(this, ky2v, &ky2)) ||
            (rc = upload_real<float>(this, kxov, &kxo)) || (rc = upload_real<float>(this, kyov, &kyo)) ||
            (rc = upload_real<float>(this, kpx, &keepx)) || (rc = upload_real<float>(this, kpy, &keepy)))
            return rc;
    } else {
        if ((rc = upload_real<double>(this, kx2v, &kx2)) || (rc = upload_real<double>(this, ky2v, &ky2)) ||
            (rc = upload_real<double>(this, kxov, &kxo)) || (rc = upload_real<double>(this, kyov, &kyo)) ||
            (rc = upload_real<double>(this, kpx, &keepx)) || (rc = upload_real<double>(this, kpy, &keepy)))
            return rc;
    }
    if (p.eq == PSS_EQ_NS && p.rfft) {
        ns_half = true;
        nsx = nx / 2 + 8;  // a multiple of every column-tile width
    }
    if (p.eq == PSS_EQ_SG && p.rfft) {
        half = true;
        sx = nx / 2 + 8;  // a multiple of every column-tile width
        const size_t hb = size_t(sx) * size_t(ny) * size_t(batch) * esz;
        for (int i = 0; i < 3; ++i) {
            if ((rc = alloc(&hbuf[i], hb))) return rc;
            if ((rc = cuda(cudaMemset(hbuf[i], 0, hb), "memset"))) return rc;
        }
        if ((rc = upload_twiddles(this, nx / 2, &twm))) return rc;
        std::vector<double> kh(sx, 0.0);
        for (int64_t m = 0; m <= nx / 2; ++m) kh[m] = kx2v[m];
        if ((rc = p.precision == PSS_FP32 ? upload_real<float>(this, kh, &kx2h) : upload_real<double>(this, kh, &kx2h)))
            return rc;
    }
    if (p.eq == PSS_EQ_NLS) {
        // exp(-i k^2 tau) - 1 = (-2 sin^2(k^2 tau / 2), -sin(k^2 tau)) per axis,
        // tau = dt/2 (index 0) and dt (index 1); no cancellation for small k
        for (int h = 0; h < 2; ++h) {
            const double tau = h == 0 ? 0.5 * p.dt : p.dt;
            auto km1 = [](double ph, double *re, double *im) {
                const double sh = std::sin(0.5 * ph);
                *re = -2.0 * sh * sh;
                *im = -std::sin(ph);
            };
            auto fx = [&](int64_t m, double *re, double *im) { km1(kx2v[m] * tau, re, im); };
            auto fy = [&](int64_t m, double *re, double *im) { km1(ky2v[m] * tau, re, im); };
            if ((rc = upload_cplx_table(this, nx, fx, &ax[h]))) return rc;
            if ((rc = upload_cplx_table(this, ny, fy, &by[h]))) return rc;
        }
    }
    // reductions
    const size_t parts = size_t(batch) * 3 * std::max<int64_t>(RED_BLOCKS, nx);
    if ((rc = alloc((void **)&partials, parts * 8))) return rc;
    if ((rc = alloc((void **)&sums, size_t(batch) * 3 * 8))) return rc;
    // NS: the per-tile words of the split column pass follow the 64-byte block
    const size_t flag_bytes = 64 + (p.eq == PSS_EQ_NS ? size_t(batch) * size_t(nx) * 4 : 0);
    if ((rc = alloc((void **)&flags, flag_bytes))) return rc;
    if ((rc = cuda(cudaMemset(flags, 0, flag_bytes), "memset"))) return rc;
    void *hp = nullptr;
    if ((rc = cuda(cudaMallocHost(&hp, size_t(batch) * 3 * 8 + 64), "cudaMallocHost"))) return rc;
    owned_host.push_back(hp);
    host_sums = static_cast<double *>(hp);
    host_flags = reinterpret_cast<unsigned *>(static_cast<char *>(hp) + size_t(batch) * 3 * 8);
    if (p.eq == PSS_EQ_NS) {
        if ((rc = alloc(&ns_field, size_t(batch) * ns_field_bytes()))) return rc;
        if ((rc = cuda(cudaMemset(ns_field, 0, size_t(batch) * ns_field_bytes()), "memset"))) return rc;
        if ((rc = cuda(cudaMallocHost(&hp, size_t(batch) * ns_field_bytes()), "cudaMallocHost"))) return rc;
        owned_host.push_back(hp);
        host_fields = hp;
    }
    return cuda(cudaDeviceSynchronize(), "init sync");
}

int pss_grid::sync()
{
    int rc = cuda(cudaStreamSynchronize(stream), "stream sync");
    if (rc) return rc;
    if ((rc = check_pass_status())) return rc;
    if ((rc = check_ns_nonconv())) return rc;
    if (nonconv_pending) {
        nonconv_pending = false;
        return fail(PSS_E_NOT_CONVERGED, "NS fixed point reached max_iter=%d", p.max_iter);
    }
    return PSS_OK;
}

namespace pss {
PlanTuning *plan_tuning()
{
    thread_local PlanTuning t;
    return &t;
}
std::atomic<int> &plan_epoch()
{
    static std::atomic<int> e{0};
    return e;
}
}  // namespace pss

int pss_grid::pass_begin(int kind)
{
    ++launches;
    plan_tuning()->open_kind = kind;
    if (!profiling) return PSS_OK;
    prof_open = sampled(prof_pass++);
    if (!prof_open) return PSS_OK;
    if (capturing) {
        // a profiling graph: an event pair around each timed pass; the graph
        // owns its events
        cudaEvent_t e;
        int rc = cuda(cudaEventCreate(&e), "event create");
        if (rc) return rc;
        capturing->evs.push_back(e);
        capturing->kinds.push_back(kind);
        // External: a node of the graph that records the event when it runs
        // (a plain record during capture only orders the captured work)
        return cuda(cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal), "event record");
    }
    while (ev_pool.size() < ev_used + 2) {
        cudaEvent_t e;
        int rc = cuda(cudaEventCreate(&e), "event create");
        if (rc) return rc;
        ev_pool.push_back(e);
    }
    ev_kind.push_back(kind);
    return cuda(cudaEventRecord(ev_pool[ev_used++], stream), "event record");
}

int pss_grid::pass_end()
{
    plan_tuning()->open_kind = -1;
    if (!profiling || !prof_open) return PSS_OK;
    prof_open = false;
    if (capturing) {
        cudaEvent_t e;
        int rc = cuda(cudaEventCreate(&e), "event create");
        if (rc) return rc;
        capturing->evs.push_back(e);
        return cuda(cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal), "event record");
    }
    return cuda(cudaEventRecord(ev_pool[ev_used++], stream), "event record");
}

int pss_grid::profile_resolve()
{
    int rc = cuda(cudaStreamSynchronize(stream), "profile sync");
    if (rc) return rc;
    if (prof_pending) {
        // timed pass i of the graph ran between its events 2i and 2i + 1
        const StepGraph &g = *prof_pending;
        prof_pending = nullptr;
        for (size_t i = 0; i < g.kinds.size() && 2 * i + 1 < g.evs.size(); ++i) {
            float ms = 0.f;
            if ((rc = cuda(cudaEventElapsedTime(&ms, g.evs[2 * i], g.evs[2 * i + 1]), "elapsed"))) return rc;
            prof_ms[g.kinds[i]] += ms;
            prof_n[g.kinds[i]] += 1;
        }
    }
    for (size_t i = 0; i < ev_kind.size(); ++i) {
        float ms = 0.f;
        if ((rc = cuda(cudaEventElapsedTime(&ms, ev_pool[2 * i], ev_pool[2 * i + 1]), "elapsed"))) return rc;
        prof_ms[ev_kind[i]] += ms;
        prof_n[ev_kind[i]] += 1;
    }
    ev_kind.clear();
    ev_used = 0;
    return PSS_OK;
}

// per-field fixed-point record as written by the NS kernels
struct NsFieldHost {
    int idx, active, nonconv, pad;
    long long updates;
};

int pss_grid::ns_update_count(int64_t *n)
{
    *n = 0;
    if (p.eq != PSS_EQ_NS || !has_state) return PSS_OK;
    int rc = cuda(cudaMemcpyAsync(host_fields, ns_field, size_t(batch) * ns_field_bytes(), cudaMemcpyDeviceToHost,
                                  stream), "fields copy");
    if (rc || (rc = cuda(cudaStreamSynchronize(stream), "sync"))) return rc;
    const NsFieldHost *f = static_cast<const NsFieldHost *>(host_fields);
    for (int64_t i = 0; i < batch; ++i) *n += f[i].updates;
    return PSS_OK;
}

// Report (and clear) fields that reached max_iter since the last check.
// a pass kernel that gave up waiting for a tile copy left its tiles
// unfinished: the state is no longer valid
int pss_grid::check_pass_status()
{
    int *dev_slot = reinterpret_cast<int *>(flags) + pss::FLAG_SLOT_PASS_STATUS;
    int *host_slot = reinterpret_cast<int *>(host_flags) + pss::FLAG_SLOT_PASS_STATUS;
    int rc = cuda(cudaMemcpyAsync(host_slot, dev_slot, sizeof(int), cudaMemcpyDeviceToHost, stream), "status copy");
    if (rc || (rc = cuda(cudaStreamSynchronize(stream), "sync"))) return rc;
    if (*host_slot == 0) return PSS_OK;
    *host_slot = 0;
    if ((rc = cuda(cudaMemsetAsync(dev_slot, 0, sizeof(int), stream), "status reset"))) return rc;
    has_state = false;
    drop_graphs();  // captured launches are rebuilt by the next step
    return fail(PSS_E_CUDA, "a column-pass tile copy did not arrive in time; the state is lost (set it again)");
}

int pss_grid::check_ns_nonconv()
{
    if (p.eq != PSS_EQ_NS || !has_state) return PSS_OK;
    const size_t bytes = size_t(batch) * ns_field_bytes();
    int rc = cuda(cudaMemcpyAsync(host_fields, ns_field, bytes, cudaMemcpyDeviceToHost, stream), "fields copy");
    if (rc || (rc = cuda(cudaStreamSynchronize(stream), "sync"))) return rc;
    NsFieldHost *h = static_cast<NsFieldHost *>(host_fields);
    bool nc = false;
    for (int64_t i = 0; i < batch; ++i) {
        nc = nc || h[i].nonconv;
        h[i].nonconv = 0;
    }
    if (!nc) return PSS_OK;
    if ((rc = cuda(cudaMemcpyAsync(ns_field, h, bytes, cudaMemcpyHostToDevice, stream), "fields copy")) ||
        (rc = cuda(cudaStreamSynchronize(stream), "sync")))
        return rc;
    return fail(PSS_E_NOT_CONVERGED, "NS fixed point reached max_iter=%d", p.max_iter);
}

// ----------------------------------------------------------------------------
// NLS: state buf[0] = row transform of psi (unnormalised); buf[1], buf[2] scratch.

namespace {

template <class Rl> int nls_set(pss_grid *g, const void *a, int where)
{
    int rc = g->cuda(cudaMemcpyAsync(g->buf[0], a, g->field_bytes(), kind_in(where), g->stream), "set_state copy");
    if (rc) return rc;
    rc = g->cuda(fft_rows<Rl>(B<Rl>(g, 0), g->nx, g->batch * g->ny, -1, Rl(1), Tw<Rl>(g->twx), g->stream),
                 "set_state row fft");
    if (rc) return rc;
    if (where == PSS_HOST) return g->cuda(cudaStreamSynchronize(g->stream), "set_state sync");
    return PSS_OK;
}

template <class Rl> int nls_step(pss_grid *g, int64_t n)
{
    const Rl s_mid = Rl(1.0 / (double(g->nx) * double(g->ny)));  // exact: powers of two
    const Rl s_end = Rl(1.0 / double(g->ny));
    const Rl sdt = Rl(g->p.sigma * g->p.dt);
    auto col = [&](int full, Rl scale) {
        return nls_col_pass<Rl>(B<Rl>(g, 0), g->nx, g->ny, g->batch, scale, Tw<Rl>(g->ax[full]),
                                Tw<Rl>(g->by[full]), Tw<Rl>(g->twy), pass_status(g), g->stream);
    };
    if (n == 0) return PSS_OK;
    int rc;
    if ((rc = g->pass_begin(1))) return rc;
    cudaError_t e = col(0, s_mid);
    if ((rc = g->pass_end())) return rc;
    for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
        if ((rc = g->pass_begin(0))) return rc;
        e = nls_row_pass<Rl>(B<Rl>(g, 0), g->nx, g->batch * g->ny, sdt, Tw<Rl>(g->twx), g->stream);
        if ((rc = g->pass_end())) return rc;
        if (e != cudaSuccess) break;
        const bool last = (i + 1 == n);
        if ((rc = g->pass_begin(1))) return rc;
        e = col(last ? 0 : 1, last ? s_end : s_mid);
        if ((rc = g->pass_end())) return rc;
    }
    return g->cuda(e, "nls step");
}

// psi (physical) into buf[1]
template <class Rl> int nls_physical(pss_grid *g)
{
    int rc = g->cuda(cudaMemcpyAsync(g->buf[1], g->buf[0], g->field_bytes(), cudaMemcpyDeviceToDevice, g->stream),
                     "copy");
    if (rc) return rc;
    return g->cuda(fft_rows<Rl>(B<Rl>(g, 1), g->nx, g->batch * g->ny, +1, Rl(1.0 / double(g->nx)),
                                Tw<Rl>(g->twx), g->stream),
                   "row inverse");
}

template <class Rl> int nls_get(pss_grid *g, void *a, int where)
{
    int rc = nls_physical<Rl>(g);
    if (rc) return rc;
    rc = g->cuda(cudaMemcpyAsync(a, g->buf[1], g->field_bytes(), kind_out(where), g->stream), "get_state copy");
    if (rc) return rc;
    return g->sync();
}

template <class Rl> int nls_conserved(pss_grid *g, double *out)
{
    int rc = nls_physical<Rl>(g);
    if (rc) return rc;
    rc = g->cuda(cudaMemcpyAsync(g->buf[2], g->buf[0], g->field_bytes(), cudaMemcpyDeviceToDevice, g->stream),
                 "copy");
    if (rc) return rc;
    rc = g->cuda(fft_cols<Rl>(B<Rl>(g, 2), g->nx, g->ny, g->batch, -1, Rl(1), Tw<Rl>(g->twy), g->stream),
                 "col fft");
    if (rc) return rc;
    rc = g->cuda(nls_sums<Rl>(B<Rl>(g, 1), B<Rl>(g, 2), g->nx, g->ny, g->batch, g->kx2d, g->ky2d, g->partials,
                              g->sums, g->stream),
                 "nls sums");
    if (rc) return rc;
    rc = g->cuda(cudaMemcpyAsync(g->host_sums, g->sums, size_t(g->batch) * 3 * 8, cudaMemcpyDeviceToHost, g->stream),
                 "sums copy");
    if (rc) return rc;
    if ((rc = g->sync())) return rc;
    const double dA = g->dA(), inv_n = 1.0 / (double(g->nx) * double(g->ny));
    bool finite = true;
    for (int64_t f = 0; f < g->batch; ++f) {
        const double *s = g->host_sums + 3 * f;
        out[2 * f] = dA * s[0];
        out[2 * f + 1] = dA * (0.5 * s[2] * inv_n + 0.25 * g->p.sigma * s[1]);
        finite = finite && std::isfinite(out[2 * f]) && std::isfinite(out[2 * f + 1]);
    }
    return finite ? PSS_OK : g->fail(PSS_E_NONFINITE, "non-finite NLS invariant");
}

}  // namespace

// ----------------------------------------------------------------------------
// shared helpers

namespace {

// forward (-1) or inverse (+1, with 1/(nx ny)) 2D transform of buffer b
template <class Rl> cudaError_t fft2(pss_grid *g, V2<Rl> *b, int dir)
{
    cudaError_t e = fft_rows<Rl>(b, g->nx, g->batch * g->ny, dir, Rl(1), Tw<Rl>(g->twx), g->stream);
    if (e != cudaSuccess) return e;
    const Rl sc = dir > 0 ? Rl(1.0 / (double(g->nx) * double(g->ny))) : Rl(1);
    return fft_cols<Rl>(b, g->nx, g->ny, g->batch, dir, sc, Tw<Rl>(g->twy), g->stream);
}

// real caller array (host or device) -> complex buffer dst (imaginary part 0),
// through the raw scratch buffer `tmp`
template <class Rl> int load_real(pss_grid *g, const void *src, int where, int tmp, int dst, bool apply_sin)
{
    const size_t bytes = size_t(g->ntot) * sizeof(Rl);
    int rc = g->cuda(cudaMemcpyAsync(g->buf[tmp], src, bytes, kind_in(where), g->stream), "state copy");
    if (rc) return rc;
    return g->cuda(real_to_complex<Rl>(static_cast<const Rl *>(g->buf[tmp]), B<Rl>(g, dst), g->ntot, apply_sin,
                                       g->stream), "real to complex");
}

// Re(a - c b) of complex buffers into the caller array (through `tmp` for HOST)
template <class Rl>
int store_real(pss_grid *g, const V2<Rl> *a, const V2<Rl> *b, Rl c, void *dst, int where, int tmp)
{
    Rl *d = where == PSS_DEVICE ? static_cast<Rl *>(dst) : static_cast<Rl *>(g->buf[tmp]);
    int rc = g->cuda(complex_to_real<Rl>(a, b, c, d, g->ntot, g->stream), "complex to real");
    if (rc || where == PSS_DEVICE) return rc;
    return g->cuda(cudaMemcpyAsync(dst, d, size_t(g->ntot) * sizeof(Rl), cudaMemcpyDeviceToHost, g->stream),
                   "state copy");
}

template <class Rl> const Rl *Rt(const void *p) { return static_cast<const Rl *>(p); }

int finish_sums(pss_grid *g)
{
    int rc = g->cuda(cudaMemcpyAsync(g->host_sums, g->sums, size_t(g->batch) * 3 * 8, cudaMemcpyDeviceToHost,
                                     g->stream), "sums copy");
    return rc ? rc : g->sync();
}

}  // namespace

// ----------------------------------------------------------------------------
// Sine-Gordon: buf[0] = uhat^n, buf[1] = d^n = uhat^n - uhat^{n-1},
// buf[2] = H (column inverse transform of uhat^n / (nx ny)); buf[3], buf[4] scratch.

namespace {

// H from uhat: the same scaling-then-transform as the fused column pass
template <class Rl> int sg_make_h(pss_grid *g)
{
    const Rl s = Rl(1.0 / (double(g->nx) * double(g->ny)));  // power of two: exact before or after
    int rc = g->cuda(cudaMemcpyAsync(g->buf[2], g->buf[0], g->field_bytes(), cudaMemcpyDeviceToDevice, g->stream),
                     "copy");
    if (rc) return rc;
    return g->cuda(fft_cols<Rl>(B<Rl>(g, 2), g->nx, g->ny, g->batch, +1, s, Tw<Rl>(g->twy), g->stream), "H");
}

// both levels from u^n, u^{n-1}: uhat^n = F u^n, d = uhat^n - F u^{n-1}
template <class Rl> int sg_set_levels(pss_grid *g, const void *un, const void *unm1, int where)
{
    int rc;
    if ((rc = load_real<Rl>(g, un, where, 3, 0, false)) || (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 0), -1), "forward")) ||
        (rc = load_real<Rl>(g, unm1, where, 3, 1, false)) || (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 1), -1), "forward")) ||
        (rc = g->cuda(cplx_axpy<Rl>(B<Rl>(g, 0), B<Rl>(g, 1), Rl(1), B<Rl>(g, 1), g->ntot, g->stream), "d")) ||
        (rc = sg_make_h<Rl>(g)))
        return rc;
    return where == PSS_HOST ? g->cuda(cudaStreamSynchronize(g->stream), "sync") : PSS_OK;
}

// half spectra <-> full spectra of the sine-Gordon state
template <class Rl> int sg_half_sync(pss_grid *g, bool to_half)
{
    int rc;
    V2<Rl> *hu = static_cast<V2<Rl> *>(g->hbuf[0]), *hd = static_cast<V2<Rl> *>(g->hbuf[1]),
           *hh = static_cast<V2<Rl> *>(g->hbuf[2]);
    if (to_half) {
        const size_t hb = size_t(g->sx) * size_t(g->ny) * size_t(g->batch) * g->esz;
        const Rl s = Rl(1.0 / (double(g->nx) * double(g->ny)));
        if ((rc = g->cuda(pack_half<Rl>(B<Rl>(g, 0), hu, g->nx, g->ny, g->sx, g->batch, g->stream), "pack")) ||
            (rc = g->cuda(pack_half<Rl>(B<Rl>(g, 1), hd, g->nx, g->ny, g->sx, g->batch, g->stream), "pack")) ||
            (rc = g->cuda(cudaMemcpyAsync(hh, hu, hb, cudaMemcpyDeviceToDevice, g->stream), "copy")) ||
            (rc = g->cuda(fft_cols<Rl>(hh, g->sx, g->ny, g->batch, +1, s, Tw<Rl>(g->twy), g->stream), "H")))
            return rc;
        return PSS_OK;
    }
    if ((rc = g->cuda(unpack_half<Rl>(hu, B<Rl>(g, 0), g->nx, g->ny, g->sx, g->batch, g->stream), "unpack")) ||
        (rc = g->cuda(unpack_half<Rl>(hd, B<Rl>(g, 1), g->nx, g->ny, g->sx, g->batch, g->stream), "unpack")))
        return rc;
    return PSS_OK;
}

template <class Rl> int sg_set(pss_grid *g, const void *u0, const void *v0, int where)
{
    int rc;
    if ((rc = load_real<Rl>(g, u0, where, 3, 0, false))) return rc;
    if ((rc = g->cuda(real_to_complex<Rl>(static_cast<const Rl *>(g->buf[3]), B<Rl>(g, 2), g->ntot, true, g->stream),
                      "sin u0")))
        return rc;
    if (v0) {
        if ((rc = load_real<Rl>(g, v0, where, 3, 1, false))) return rc;
    } else if ((rc = g->cuda(cudaMemsetAsync(g->buf[1], 0, g->field_bytes(), g->stream), "memset"))) {
        return rc;
    }
    for (int b : {0, 1, 2})
        if ((rc = g->cuda(fft2<Rl>(g, B<Rl>(g, b), -1), "forward transform"))) return rc;
    if ((rc = g->cuda(sg_init<Rl>(B<Rl>(g, 0), B<Rl>(g, 1), B<Rl>(g, 2), g->kx2d, g->ky2d, g->p.dt, g->nx, g->ny,
                                  g->batch, g->stream), "sg init")))
        return rc;
    if ((rc = sg_make_h<Rl>(g))) return rc;
    return where == PSS_HOST ? g->cuda(cudaStreamSynchronize(g->stream), "sync") : PSS_OK;
}

template <class Rl> int sg_step(pss_grid *g, int64_t n)
{
    int rc;
    if (g->half) {
        V2<Rl> *u = static_cast<V2<Rl> *>(g->hbuf[0]), *d = static_cast<V2<Rl> *>(g->hbuf[1]),
               *h = static_cast<V2<Rl> *>(g->hbuf[2]);
        for (int64_t i = 0; i < n; ++i) {
            if ((rc = g->pass_begin(0))) return rc;
            cudaError_t e = sg_row_pass_r2c<Rl>(h, g->nx, g->sx, g->batch * g->ny, Tw<Rl>(g->twm), Tw<Rl>(g->twx),
                                                g->stream);
            if ((rc = g->pass_end()) || (rc = g->cuda(e, "sg row pass (half spectrum)"))) return rc;
            if ((rc = g->pass_begin(1))) return rc;
            e = sg_col_pass<Rl>(h, u, d, g->sx, g->ny, g->batch, Rt<Rl>(g->kx2h), Rt<Rl>(g->ky2), Rl(g->p.dt),
                                Tw<Rl>(g->twy), pass_status(g), g->stream, g->nx);
            if ((rc = g->pass_end()) || (rc = g->cuda(e, "sg column pass (half spectrum)"))) return rc;
        }
        return PSS_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        if ((rc = g->pass_begin(0))) return rc;
        cudaError_t e = sg_row_pass<Rl>(B<Rl>(g, 2), g->nx, g->batch * g->ny, Tw<Rl>(g->twx), g->stream);
        if ((rc = g->pass_end()) || (rc = g->cuda(e, "sg row pass"))) return rc;
        if ((rc = g->pass_begin(1))) return rc;
        e = sg_col_pass<Rl>(B<Rl>(g, 2), B<Rl>(g, 0), B<Rl>(g, 1), g->nx, g->ny, g->batch, Rt<Rl>(g->kx2),
                            Rt<Rl>(g->ky2), Rl(g->p.dt), Tw<Rl>(g->twy), pass_status(g), g->stream);
        if ((rc = g->pass_end()) || (rc = g->cuda(e, "sg column pass"))) return rc;
    }
    return PSS_OK;
}

// u^n -> a, u^{n-1} = Re F^-1 (uhat - d) -> b
template <class Rl> int sg_get(pss_grid *g, void *a, void *b, int where)
{
    int rc;
    if ((rc = g->cuda(cudaMemcpyAsync(g->buf[3], g->buf[0], g->field_bytes(), cudaMemcpyDeviceToDevice, g->stream),
                      "copy")) ||
        (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 3), +1), "inverse")) ||
        (rc = store_real<Rl>(g, B<Rl>(g, 3), nullptr, Rl(0), a, where, 4)))
        return rc;
    if (b) {
        if ((rc = g->cuda(cplx_axpy<Rl>(B<Rl>(g, 0), B<Rl>(g, 1), Rl(1), B<Rl>(g, 3), g->ntot, g->stream), "axpy")) ||
            (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 3), +1), "inverse")) ||
            (rc = store_real<Rl>(g, B<Rl>(g, 3), nullptr, Rl(0), b, where, 4)))
            return rc;
    }
    return g->sync();
}

template <class Rl> int sg_conserved(pss_grid *g, double *out)
{
    int rc;
    for (int k : {0, 1}) {
        if ((rc = g->cuda(cudaMemcpyAsync(g->buf[3 + k], g->buf[k], g->field_bytes(), cudaMemcpyDeviceToDevice,
                                          g->stream), "copy")) ||
            (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 3 + k), +1), "inverse")))
            return rc;
    }
    if ((rc = g->cuda(sg_sums<Rl>(B<Rl>(g, 3), B<Rl>(g, 4), B<Rl>(g, 0), B<Rl>(g, 1), g->nx, g->ny, g->batch, g->kx2d,
                                  g->ky2d, g->p.dt, g->partials, g->sums, g->stream), "sg sums")) ||
        (rc = finish_sums(g)))
        return rc;
    const double dA = g->dA(), inv_n = 1.0 / (double(g->nx) * double(g->ny));
    bool finite = true;
    for (int64_t f = 0; f < g->batch; ++f) {
        const double *s = g->host_sums + 3 * f;
        out[f] = dA * (s[0] + s[1]) + 0.5 * dA * s[2] * inv_n;
        finite = finite && std::isfinite(out[f]);
    }
    return finite ? PSS_OK : g->fail(PSS_E_NONFINITE, "non-finite SG Hamiltonian");
}

}  // namespace

// ----------------------------------------------------------------------------
// Navier-Stokes: buf[0..2] vorticity iterates (per-field index in ns_field),
// buf[3] = J_hat^n, buf[4] = C1, buf[5] = C2, buf[6] scratch.

namespace {

// buffer i of field f
template <class Rl> V2<Rl> *Bf(pss_grid *g, int i, int64_t f) { return B<Rl>(g, i) + f * g->npts; }

template <class Rl> void ns_w(pss_grid *g, V2<Rl> *w[3])
{
    for (int i = 0; i < 3; ++i) w[i] = B<Rl>(g, i);
}

// derivatives of w^n into C1, C2 (per_step: w^n of each field in its own
// buffer idx; otherwise in buffer 0, as after set_state)
template <class Rl> int ns_prep(pss_grid *g, bool per_step = false)
{
    V2<Rl> *w[3];
    ns_w<Rl>(g, w);
    return g->cuda(ns_prep_pass<Rl>(w, per_step ? g->ns_field : nullptr, B<Rl>(g, 4), B<Rl>(g, 5), Rt<Rl>(g->kxo),
                                    Rt<Rl>(g->kyo), Rt<Rl>(g->kx2), Rt<Rl>(g->ky2), g->nx, g->ny, g->batch,
                                    Tw<Rl>(g->twy), g->stream, g->ns_half ? g->nsx : 0), "ns derivatives");
}

// offset of field f in a vorticity buffer (half spectra: rows of nsx)
inline int64_t ns_off(const pss_grid *g, int64_t f) { return f * g->ny * (g->ns_half ? g->nsx : g->nx); }

// derivatives of field f alone (its w^n in buffer 0)
template <class Rl> int ns_prep_one(pss_grid *g, int64_t f)
{
    V2<Rl> *w[3] = {B<Rl>(g, 0) + ns_off(g, f), B<Rl>(g, 1) + ns_off(g, f), B<Rl>(g, 2) + ns_off(g, f)};
    return g->cuda(ns_prep_pass<Rl>(w, nullptr, Bf<Rl>(g, 4, f), Bf<Rl>(g, 5, f), Rt<Rl>(g->kxo), Rt<Rl>(g->kyo),
                                    Rt<Rl>(g->kx2), Rt<Rl>(g->ky2), g->nx, g->ny, 1, Tw<Rl>(g->twy), g->stream,
                                    g->ns_half ? g->nsx : 0),
                   "ns derivatives");
}

// half spectra: the full spectra of `batch` fields at src into the vorticity
// layout at dst (through buf[6] when src is buf[0] itself)
template <class Rl> int ns_to_half(pss_grid *g, V2<Rl> *src, V2<Rl> *dst, int64_t batch)
{
    if (src == dst) {
        const size_t hb = size_t(g->nsx) * size_t(g->ny) * size_t(batch) * g->esz;
        int rc = g->cuda(pack_half<Rl>(src, B<Rl>(g, 6), g->nx, g->ny, g->nsx, batch, g->stream), "pack");
        if (rc) return rc;
        return g->cuda(cudaMemcpyAsync(dst, B<Rl>(g, 6), hb, cudaMemcpyDeviceToDevice, g->stream), "copy");
    }
    return g->cuda(pack_half<Rl>(src, dst, g->nx, g->ny, g->nsx, batch, g->stream), "pack");
}

// start of a step: mark every field active; the midpoint scheme also needs
// the derivatives of w^n (its last column pass wrote those of the midpoint)
template <class Rl> int ns_step_begin(pss_grid *g)
{
    int rc = g->cuda(ns_begin(g->ns_field, g->batch, reinterpret_cast<int *>(g->flags), g->stream), "ns begin");
    if (!rc && g->p.scheme == PSS_NS_MIDPOINT) rc = ns_prep<Rl>(g, true);
    return rc;
}

template <class Rl> int ns_set(pss_grid *g, const void *w0, int where)
{
    int rc;
    if ((rc = load_real<Rl>(g, w0, where, 6, 0, false)) || (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 0), -1), "forward")) ||
        (rc = g->cuda(apply_mask<Rl>(B<Rl>(g, 0), Rt<Rl>(g->keepx), Rt<Rl>(g->keepy), g->nx, g->ny, g->batch, g->stream),
                      "mask")) ||
        (rc = g->cuda(cudaMemsetAsync(g->ns_field, 0, size_t(g->batch) * ns_field_bytes(), g->stream), "memset")) ||
        (g->ns_half && (rc = ns_to_half<Rl>(g, B<Rl>(g, 0), B<Rl>(g, 0), g->batch))) || (rc = ns_prep<Rl>(g)))
        return rc;
    return where == PSS_HOST ? g->cuda(cudaStreamSynchronize(g->stream), "sync") : PSS_OK;
}

// the passes of one fixed-point update (row pass, column pass, decide, advance)
template <class Rl> int ns_update(pss_grid *g, bool in_graph)
{
    V2<Rl> *w[3];
    ns_w<Rl>(g, w);
    int *ctl = reinterpret_cast<int *>(g->flags);
    const double parseval = g->p.lx * g->p.ly / (double(g->npts) * double(g->npts));
    int rc;
    if (!in_graph && (rc = g->pass_begin(0))) return rc;
    cudaError_t e = ns_row_pass<Rl>(B<Rl>(g, 4), B<Rl>(g, 5), g->ns_field, g->nx, g->ny, g->batch,
                                    Tw<Rl>(g->twx), g->stream, g->p.dealias != 0, g->ns_half);
    if ((!in_graph && (rc = g->pass_end())) || (rc = g->cuda(e, "ns row pass"))) return rc;
    int groups = 0;
    if (!in_graph && (rc = g->pass_begin(1))) return rc;
    e = ns_col_pass<Rl>(B<Rl>(g, 4), B<Rl>(g, 5), w, B<Rl>(g, 3), g->ns_field, g->partials, Rt<Rl>(g->kxo),
                        Rt<Rl>(g->kyo), Rt<Rl>(g->kx2), Rt<Rl>(g->ky2), Rt<Rl>(g->keepx), Rt<Rl>(g->keepy), g->p.dt,
                        g->p.nu, g->nx, g->ny, g->batch, ctl, g->p.scheme == PSS_NS_MIDPOINT ? 1 : 0, Tw<Rl>(g->twy),
                        &groups, g->stream, g->p.dealias != 0, g->ns_half ? g->nsx : 0);
    if ((!in_graph && (rc = g->pass_end())) || (rc = g->cuda(e, "ns column pass"))) return rc;
    if (!in_graph && (rc = g->pass_begin(2))) return rc;
    e = ns_decide(g->ns_field, g->partials, groups, g->batch, ctl, parseval, g->p.tol, g->p.max_iter, g->stream);
    if (e == cudaSuccess) e = ns_advance(ctl, in_graph, g->ns_cond, g->stream);
    if ((!in_graph && (rc = g->pass_end())) || (rc = g->cuda(e, "ns decide"))) return rc;
    return PSS_OK;
}

// One step as a graph: begin (and, midpoint scheme, the derivatives of w^n),
// then WHILE(some field active) { one update }.
template <class Rl> int ns_build_graph(pss_grid *g)
{
    cudaGraph_t graph = nullptr;
    int rc;
    if ((rc = g->cuda(cudaGraphCreate(&graph, 0), "graph create"))) return rc;
    g->ns_graph = graph;
    if ((rc = g->cuda(cudaGraphConditionalHandleCreate(&g->ns_cond, graph, 1, cudaGraphCondAssignDefault),
                      "conditional handle")))
        return rc;
    if ((rc = g->cuda(cudaStreamBeginCaptureToGraph(g->stream, graph, nullptr, nullptr, 0,
                                                    cudaStreamCaptureModeRelaxed), "capture")))
        return rc;
    rc = ns_step_begin<Rl>(g);
    // the last node captured so far: the WHILE node depends on it
    cudaGraphNode_t begin_node = nullptr;
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(g->stream, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess && ndeps == 1) begin_node = deps[0];
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(g->stream, &out);
    if (rc) return rc;
    if ((rc = g->cuda(e != cudaSuccess ? e : e2, "capture begin"))) return rc;
    if (!begin_node) return g->fail(PSS_E_CUDA, "step graph: expected one node before the loop, found %zu", ndeps);
    // zero-initialised node parameters (the struct's union has no default constructor)
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = g->ns_cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if ((rc = g->cuda(cudaGraphAddNode(&cnode, graph, &begin_node, nullptr, 1, &cp), "conditional node"))) return rc;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((rc = g->cuda(cudaStreamBeginCaptureToGraph(g->stream, body, nullptr, nullptr, 0,
                                                    cudaStreamCaptureModeRelaxed), "capture body")))
        return rc;
    rc = ns_update<Rl>(g, true);
    e2 = cudaStreamEndCapture(g->stream, &out);
    if (rc) return rc;
    if ((rc = g->cuda(e2, "capture body end"))) return rc;
    return g->cuda(cudaGraphInstantiate(&g->ns_exec, graph, 0), "graph instantiate");
}

template <class Rl> int ns_step(pss_grid *g, int64_t n)
{
    int *ctl = reinterpret_cast<int *>(g->flags);
    int *hctl = reinterpret_cast<int *>(g->host_flags);
    int rc;
    if (g->use_graphs && !g->profiling && !g->ns_exec && ns_build_graph<Rl>(g) != PSS_OK) {
        // capture is not available here: keep stepping with direct launches
        g->use_graphs = false;
        cudaGetLastError();
        g->err.clear();
    }
    if (g->use_graphs && !g->profiling) {
        for (int64_t s = 0; s < n; ++s)
            if ((rc = g->cuda(cudaGraphLaunch(g->ns_exec, g->stream), "graph launch"))) return rc;
        return PSS_OK;  // a field that reached max_iter is reported by the next synchronising call
    }
    for (int64_t s = 0; s < n; ++s) {
        if ((rc = ns_step_begin<Rl>(g))) return rc;
        for (int k = 0; k < g->p.max_iter; ++k) {
            if ((rc = ns_update<Rl>(g, false))) return rc;
            if ((rc = g->cuda(cudaMemcpyAsync(hctl, ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->stream),
                              "ctl copy")) ||
                (rc = g->cuda(cudaStreamSynchronize(g->stream), "ns sync")))
                return rc;
            if (hctl[2] == 0) break;
        }
    }
    rc = g->check_ns_nonconv();
    if (rc == PSS_E_NOT_CONVERGED) g->steps += n;  // the steps were taken; pss_grid::step_n adds n only on success
    return rc;
}

// current vorticity of every field into buf[6] (full spectra); half
// spectra gather into buf[3] (J_hat^n, rebuilt at the start of every step)
// and are extended to full width
template <class Rl> int ns_current(pss_grid *g)
{
    V2<Rl> *w[3];
    ns_w<Rl>(g, w);
    if (!g->ns_half)
        return g->cuda(ns_gather<Rl>(g->ns_field, w, B<Rl>(g, 6), g->npts, g->batch, g->stream), "gather");
    int rc = g->cuda(ns_gather<Rl>(g->ns_field, w, B<Rl>(g, 3), g->ny * g->nsx, g->batch, g->stream), "gather");
    if (rc) return rc;
    return g->cuda(unpack_half<Rl>(B<Rl>(g, 3), B<Rl>(g, 6), g->nx, g->ny, g->nsx, g->batch, g->stream), "unpack");
}

template <class Rl> int ns_get(pss_grid *g, void *a, int where)
{
    int rc;
    if ((rc = ns_current<Rl>(g)) || (rc = g->cuda(fft2<Rl>(g, B<Rl>(g, 6), +1), "inverse")) ||
        (rc = store_real<Rl>(g, B<Rl>(g, 6), nullptr, Rl(0), a, where, 3)))
        return rc;
    return g->sync();
}

template <class Rl> int ns_conserved(pss_grid *g, double *out)
{
    V2<Rl> *w[3];
    ns_w<Rl>(g, w);
    int rc;
    if (g->ns_half) {  // sums over the full spectra of buf[6]
        if ((rc = ns_current<Rl>(g))) return rc;
        w[0] = w[1] = w[2] = B<Rl>(g, 6);
    }
    if ((rc = g->cuda(ns_sums<Rl>(g->ns_field, w, g->nx, g->ny, g->batch, g->kx2d, g->ky2d, g->partials, g->sums,
                                  g->stream), "ns sums")) ||
        (rc = finish_sums(g)))
        return rc;
    const double dA = g->dA(), inv_n = 1.0 / (double(g->nx) * double(g->ny));
    bool finite = true;
    for (int64_t f = 0; f < g->batch; ++f) {
        const double *s = g->host_sums + 3 * f;
        out[3 * f] = dA * s[0];
        out[3 * f + 1] = 0.5 * dA * s[1] * inv_n;
        out[3 * f + 2] = 0.5 * dA * s[2] * inv_n;
        for (int k = 0; k < 3; ++k) finite = finite && std::isfinite(out[3 * f + k]);
    }
    return finite ? PSS_OK : g->fail(PSS_E_NONFINITE, "non-finite NS invariant");
}

}  // namespace

// ----------------------------------------------------------------------------
// One field of the batch (slot f): the set-up and read-back of the equation on
// the sub-arrays of field f, with batch 1.

namespace {

template <class Rl> cudaError_t fft2_one(pss_grid *g, V2<Rl> *b, int dir)
{
    cudaError_t e = fft_rows<Rl>(b, g->nx, g->ny, dir, Rl(1), Tw<Rl>(g->twx), g->stream);
    if (e != cudaSuccess) return e;
    const Rl sc = dir > 0 ? Rl(1.0 / (double(g->nx) * double(g->ny))) : Rl(1);
    return fft_cols<Rl>(b, g->nx, g->ny, 1, dir, sc, Tw<Rl>(g->twy), g->stream);
}

// real field (host or device) -> complex slot dst_buf[f], through raw scratch slot tmp_buf[f]
template <class Rl>
int load_real_one(pss_grid *g, int64_t f, const void *src, int where, int tmp, int dst, bool apply_sin)
{
    Rl *t = reinterpret_cast<Rl *>(Bf<Rl>(g, tmp, f));
    int rc = g->cuda(cudaMemcpyAsync(t, src, size_t(g->npts) * sizeof(Rl), kind_in(where), g->stream), "copy");
    if (rc) return rc;
    return g->cuda(real_to_complex<Rl>(t, Bf<Rl>(g, dst, f), g->npts, apply_sin, g->stream), "real to complex");
}

template <class Rl> int store_real_one(pss_grid *g, int64_t f, const V2<Rl> *a, void *dst, int where, int tmp)
{
    Rl *d = where == PSS_DEVICE ? static_cast<Rl *>(dst) : reinterpret_cast<Rl *>(Bf<Rl>(g, tmp, f));
    int rc = g->cuda(complex_to_real<Rl>(a, nullptr, Rl(0), d, g->npts, g->stream), "complex to real");
    if (rc || where == PSS_DEVICE) return rc;
    return g->cuda(cudaMemcpyAsync(dst, d, size_t(g->npts) * sizeof(Rl), cudaMemcpyDeviceToHost, g->stream), "copy");
}

template <class Rl> int field_set(pss_grid *g, int64_t f, const void *a, const void *b, int where)
{
    int rc = PSS_OK;
    const size_t fb = size_t(g->npts) * g->esz;
    if (g->p.eq == PSS_EQ_NLS) {
        if ((rc = g->cuda(cudaMemcpyAsync(Bf<Rl>(g, 0, f), a, fb, kind_in(where), g->stream), "copy")) ||
            (rc = g->cuda(fft_rows<Rl>(Bf<Rl>(g, 0, f), g->nx, g->ny, -1, Rl(1), Tw<Rl>(g->twx), g->stream), "row fft")))
            return rc;
    } else if (g->p.eq == PSS_EQ_SG) {
        if ((rc = load_real_one<Rl>(g, f, a, where, 3, 0, false)) ||
            (rc = g->cuda(real_to_complex<Rl>(reinterpret_cast<Rl *>(Bf<Rl>(g, 3, f)), Bf<Rl>(g, 2, f), g->npts, true,
                                              g->stream), "sin")))
            return rc;
        if (b) rc = load_real_one<Rl>(g, f, b, where, 3, 1, false);
        else rc = g->cuda(cudaMemsetAsync(Bf<Rl>(g, 1, f), 0, fb, g->stream), "memset");
        if (rc) return rc;
        for (int i : {0, 1, 2})
            if ((rc = g->cuda(fft2_one<Rl>(g, Bf<Rl>(g, i, f), -1), "forward"))) return rc;
        const Rl s = Rl(1.0 / (double(g->nx) * double(g->ny)));
        if ((rc = g->cuda(sg_init<Rl>(Bf<Rl>(g, 0, f), Bf<Rl>(g, 1, f), Bf<Rl>(g, 2, f), g->kx2d, g->ky2d, g->p.dt,
                                      g->nx, g->ny, 1, g->stream), "sg init")) ||
            (rc = g->cuda(cudaMemcpyAsync(Bf<Rl>(g, 2, f), Bf<Rl>(g, 0, f), fb, cudaMemcpyDeviceToDevice, g->stream),
                          "copy")) ||
            (rc = g->cuda(fft_cols<Rl>(Bf<Rl>(g, 2, f), g->nx, g->ny, 1, +1, s, Tw<Rl>(g->twy), g->stream), "H")))
            return rc;
    } else {
        // full spectrum of the field in buf[6] (half spectra) or buf[0], then
        // (half spectra) into the field's slot of the half-width buffer 0
        const int dst = g->ns_half ? 6 : 0;
        if ((rc = load_real_one<Rl>(g, f, a, where, g->ns_half ? 3 : 6, dst, false)) ||
            (rc = g->cuda(fft2_one<Rl>(g, Bf<Rl>(g, dst, f), -1), "forward")) ||
            (rc = g->cuda(apply_mask<Rl>(Bf<Rl>(g, dst, f), Rt<Rl>(g->keepx), Rt<Rl>(g->keepy), g->nx, g->ny, 1,
                                         g->stream), "mask")) ||
            (g->ns_half && (rc = ns_to_half<Rl>(g, Bf<Rl>(g, 6, f), B<Rl>(g, 0) + ns_off(g, f), 1))) ||
            (rc = g->cuda(cudaMemsetAsync(static_cast<char *>(g->ns_field) + f * ns_field_bytes(), 0, ns_field_bytes(),
                                          g->stream), "record")) ||
            (rc = ns_prep_one<Rl>(g, f)))
            return rc;
    }
    return where == PSS_HOST ? g->cuda(cudaStreamSynchronize(g->stream), "sync") : PSS_OK;
}

template <class Rl> int field_get(pss_grid *g, int64_t f, void *a, void *b, int where)
{
    int rc;
    const size_t fb = size_t(g->npts) * g->esz;
    if (g->p.eq == PSS_EQ_NLS) {
        if ((rc = g->cuda(cudaMemcpyAsync(Bf<Rl>(g, 1, f), Bf<Rl>(g, 0, f), fb, cudaMemcpyDeviceToDevice, g->stream),
                          "copy")) ||
            (rc = g->cuda(fft_rows<Rl>(Bf<Rl>(g, 1, f), g->nx, g->ny, +1, Rl(1.0 / double(g->nx)), Tw<Rl>(g->twx),
                                       g->stream), "row inverse")) ||
            (rc = g->cuda(cudaMemcpyAsync(a, Bf<Rl>(g, 1, f), fb, kind_out(where), g->stream), "copy")))
            return rc;
    } else if (g->p.eq == PSS_EQ_SG) {
        if ((rc = g->cuda(cudaMemcpyAsync(Bf<Rl>(g, 3, f), Bf<Rl>(g, 0, f), fb, cudaMemcpyDeviceToDevice, g->stream),
                          "copy")) ||
            (rc = g->cuda(fft2_one<Rl>(g, Bf<Rl>(g, 3, f), +1), "inverse")) ||
            (rc = store_real_one<Rl>(g, f, Bf<Rl>(g, 3, f), a, where, 4)))
            return rc;
        if (b && ((rc = g->cuda(cplx_axpy<Rl>(Bf<Rl>(g, 0, f), Bf<Rl>(g, 1, f), Rl(1), Bf<Rl>(g, 3, f), g->npts,
                                              g->stream), "axpy")) ||
                  (rc = g->cuda(fft2_one<Rl>(g, Bf<Rl>(g, 3, f), +1), "inverse")) ||
                  (rc = store_real_one<Rl>(g, f, Bf<Rl>(g, 3, f), b, where, 4))))
            return rc;
    } else {
        V2<Rl> *w[3];
        for (int i = 0; i < 3; ++i) w[i] = B<Rl>(g, i) + ns_off(g, f);  // field f's slot of each vorticity buffer
        const void *rec = static_cast<char *>(g->ns_field) + f * ns_field_bytes();
        if (g->ns_half) {
            V2<Rl> *h = B<Rl>(g, 3) + ns_off(g, f);
            if ((rc = g->cuda(ns_gather<Rl>(rec, w, h, g->ny * g->nsx, 1, g->stream), "gather")) ||
                (rc = g->cuda(unpack_half<Rl>(h, Bf<Rl>(g, 6, f), g->nx, g->ny, g->nsx, 1, g->stream), "unpack")))
                return rc;
        } else if ((rc = g->cuda(ns_gather<Rl>(rec, w, Bf<Rl>(g, 6, f), g->npts, 1, g->stream), "gather"))) {
            return rc;
        }
        if ((rc = g->cuda(fft2_one<Rl>(g, Bf<Rl>(g, 6, f), +1), "inverse")) ||
            (rc = store_real_one<Rl>(g, f, Bf<Rl>(g, 6, f), a, where, 3)))
            return rc;
    }
    return g->sync();
}

}  // namespace

// ----------------------------------------------------------------------------
// dispatch by equation and precision

#define PSS_BY_PRECISION(CALL) (p.precision == PSS_FP32 ? CALL(float) : CALL(double))

int pss_grid::set_state(const void *a, const void *b, int where)
{
    steps = 0;
    nonconv_pending = false;
    int rc;
#define NLS(R) nls_set<R>(this, a, where)
#define SG(R) sg_set<R>(this, a, b, where)
#define NS(R) ns_set<R>(this, a, where)
    rc = p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : p.eq == PSS_EQ_SG ? PSS_BY_PRECISION(SG) : PSS_BY_PRECISION(NS);
#undef NLS
#undef SG
#undef NS
    if (!rc) {
        has_state = true;
        full_valid = true;
        half_valid = false;
    }
    return rc;
}

int pss_grid::set_sg_levels(const void *u_n, const void *u_nm1, int where)
{
    int rc = p.precision == PSS_FP32 ? sg_set_levels<float>(this, u_n, u_nm1, where)
                                     : sg_set_levels<double>(this, u_n, u_nm1, where);
    if (rc) return rc;
    steps = 0;
    has_state = true;
    full_valid = true;
    half_valid = false;
    return PSS_OK;
}

int pss_grid::half_sync(bool to_half)
{
    if (!half || (to_half ? half_valid : full_valid)) return PSS_OK;
    int rc = p.precision == PSS_FP32 ? sg_half_sync<float>(this, to_half) : sg_half_sync<double>(this, to_half);
    if (rc) return rc;
    (to_half ? half_valid : full_valid) = true;
    return PSS_OK;
}

int pss_grid::step_n(int64_t n)
{
    if (n == 0) return PSS_OK;
    int rc;
    prof_pass = 0;
    if (graph_epoch != plan_epoch().load()) {  // a plan changed: recapture
        drop_graphs();
        graph_epoch = plan_epoch().load();
    }
    if ((rc = half_sync(true))) return rc;
    if (half) full_valid = false;
#define NLS(R) nls_step<R>(this, n)
#define SG(R) sg_step<R>(this, n)
#define NS(R) ns_step<R>(this, n)
    if (p.eq != PSS_EQ_NS && use_graphs) {
        // the whole launch sequence of step_n(n) as one graph, cached by
        // (n, profiling); a profiling graph's own events time its passes
        const int prof_key = profiling ? prof_stride : 0;
        StepGraph *sg = nullptr;
        for (auto &e : step_graphs)
            if (e.n == n && e.prof == prof_key) sg = &e;
        if (sg && sg == prof_pending && (rc = profile_resolve())) return rc;  // its events are reused
        if (!sg) {
            StepGraph fresh;
            fresh.n = n;
            fresh.prof = prof_key;
            rc = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed), "capture");
            if (!rc) {
                const int64_t saved = launches;
                if (profiling) capturing = &fresh;
                prof_pass = 0;
                int inner = p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : PSS_BY_PRECISION(SG);
                capturing = nullptr;
                fresh.passes = launches - saved;
                launches = saved;
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(stream, &graph);
                if (inner) rc = inner;
                else if ((rc = cuda(e, "capture end")) == PSS_OK)
                    rc = cuda(cudaGraphInstantiate(&fresh.exec, graph, 0), "graph instantiate");
                if (graph) cudaGraphDestroy(graph);
            }
            if (rc) {
                // capture is not available here: direct launches from now on
                free_step_graph(fresh);
                use_graphs = false;
                cudaGetLastError();
                err.clear();
                rc = p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : PSS_BY_PRECISION(SG);
                if (!rc) steps += n;
                return rc;
            }
            if (step_graphs.size() >= 4) {
                if (prof_pending) {  // resolve before the list (and the pending entry) moves
                    if ((rc = profile_resolve())) {
                        free_step_graph(fresh);
                        return rc;
                    }
                }
                free_step_graph(step_graphs.front());
                step_graphs.erase(step_graphs.begin());
            }
            if (prof_pending) {  // the vector may reallocate below
                if ((rc = profile_resolve())) {
                    free_step_graph(fresh);
                    return rc;
                }
            }
            step_graphs.push_back(std::move(fresh));
            sg = &step_graphs.back();
        }
        rc = cuda(cudaGraphLaunch(sg->exec, stream), "graph launch");
        if (!rc) {
            launches += sg->passes;
            if (sg->prof) prof_pending = sg;
        }
    } else {
        rc = p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : p.eq == PSS_EQ_SG ? PSS_BY_PRECISION(SG) : PSS_BY_PRECISION(NS);
    }
#undef NLS
#undef SG
#undef NS
    if (!rc) steps += n;
    return rc;
}

int pss_grid::get_state(void *a, void *b, int where)
{
    int rc = half_sync(false);
    if (rc) return rc;
#define NLS(R) nls_get<R>(this, a, where)
#define SG(R) sg_get<R>(this, a, b, where)
#define NS(R) ns_get<R>(this, a, where)
    return p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : p.eq == PSS_EQ_SG ? PSS_BY_PRECISION(SG) : PSS_BY_PRECISION(NS);
#undef NLS
#undef SG
#undef NS
}

int pss_grid::set_field(int64_t f, const void *a, const void *b, int where)
{
    int rc = half_sync(false);  // the other fields' full state must be current
    if (rc) return rc;
    rc = p.precision == PSS_FP32 ? field_set<float>(this, f, a, b, where) : field_set<double>(this, f, a, b, where);
    if (!rc) {
        has_state = true;
        half_valid = false;
    }
    return rc;
}

int pss_grid::get_field(int64_t f, void *a, void *b, int where)
{
    int rc = half_sync(false);
    if (rc) return rc;
    return p.precision == PSS_FP32 ? field_get<float>(this, f, a, b, where) : field_get<double>(this, f, a, b, where);
}

int pss_grid::conserved(double *out)
{
    int rc = half_sync(false);
    if (rc) return rc;
#define NLS(R) nls_conserved<R>(this, out)
#define SG(R) sg_conserved<R>(this, out)
#define NS(R) ns_conserved<R>(this, out)
    return p.eq == PSS_EQ_NLS ? PSS_BY_PRECISION(NLS) : p.eq == PSS_EQ_SG ? PSS_BY_PRECISION(SG) : PSS_BY_PRECISION(NS);
#undef NLS
#undef SG
#undef NS
}

// Checkpoint layout: the exact state buffers (NLS: row transform of psi;
// SG: uhat^n, d^n; NS: w_hat^n of every field), then {steps, NS updates}.
size_t pss_grid::checkpoint_bytes() const
{
    const int nstate = p.eq == PSS_EQ_SG ? 2 : 1;
    return size_t(nstate) * size_t(ntot) * esz + 16;
}

int pss_grid::checkpoint(void *buf_, int where, bool save)
{
    const int nstate = p.eq == PSS_EQ_SG ? 2 : 1;
    char *b = static_cast<char *>(buf_);
    int rc;
    if (save && (rc = half_sync(false))) return rc;
    int src_of[2] = {0, 1};
    if (save && p.eq == PSS_EQ_NS) {
        rc = p.precision == PSS_FP32 ? ns_current<float>(this) : ns_current<double>(this);
        if (rc) return rc;
        src_of[0] = 6;
    }
    for (int i = 0; i < nstate; ++i) {
        if (save)
            rc = cuda(cudaMemcpyAsync(b + i * field_bytes(), this->buf[src_of[i]], field_bytes(), kind_out(where), stream),
                      "checkpoint");
        else
            rc = cuda(cudaMemcpyAsync(this->buf[i], b + i * field_bytes(), field_bytes(), kind_in(where), stream),
                      "checkpoint");
        if (rc) return rc;
    }
    int64_t meta[2] = {steps, 0};
    if (save && (rc = ns_update_count(&meta[1]))) return rc;
    char *mb = b + nstate * field_bytes();
    if (save)
        rc = cuda(cudaMemcpyAsync(mb, meta, 16, where == PSS_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, stream),
                  "checkpoint meta");
    else
        rc = cuda(cudaMemcpyAsync(meta, mb, 16, where == PSS_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, stream),
                  "checkpoint meta");
    if (rc || (rc = cuda(cudaStreamSynchronize(stream), "checkpoint sync"))) return rc;
    if (!save) {
        steps = meta[0];
        if (p.eq == PSS_EQ_SG) {
            rc = p.precision == PSS_FP32 ? sg_make_h<float>(this) : sg_make_h<double>(this);
        } else if (p.eq == PSS_EQ_NS) {
            // all fields restart from buffer 0 with their update count
            NsFieldHost *h = static_cast<NsFieldHost *>(host_fields);
            for (int64_t i = 0; i < batch; ++i) h[i] = NsFieldHost{0, 0, 0, 0, i == 0 ? meta[1] : 0};
            rc = cuda(cudaMemcpyAsync(ns_field, h, size_t(batch) * ns_field_bytes(), cudaMemcpyHostToDevice, stream),
                      "fields");
            if (!rc && ns_half)
                rc = p.precision == PSS_FP32 ? ns_to_half<float>(this, B<float>(this, 0), B<float>(this, 0), batch)
                                             : ns_to_half<double>(this, B<double>(this, 0), B<double>(this, 0), batch);
            if (!rc) rc = p.precision == PSS_FP32 ? ns_prep<float>(this) : ns_prep<double>(this);
        }
        if (rc || (rc = cuda(cudaStreamSynchronize(stream), "restore sync"))) return rc;
        has_state = true;
        full_valid = true;
        half_valid = false;
    }
    return PSS_OK;
}

// ----------------------------------------------------------------------------
// Autotuner: time `steps` steps of this grid in each launch-shape variant
// (on its own state, restored afterwards; a one-step round of each first, then
// two alternating timed rounds, best of the two) and keep, per row and per
// column pass kernel, the faster variant (variant 1 must win by more than 2 %).

int pss_grid::autotune(int k, int *changed)
{
    *changed = 0;
    if (p.precision != PSS_FP32 || p.eq == PSS_EQ_NS) return PSS_OK;  // nothing tunable
    if (!has_state) return fail(PSS_E_STATE, "autotune before set_state");
    void *save = nullptr;
    const size_t bytes = checkpoint_bytes();
    if (cudaMalloc(&save, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSS_E_OOM, "autotune: no room for a copy of the state");
    }
    int rc = checkpoint(save, PSS_DEVICE, true);
    const bool prof = profiling;
    const int stride = prof_stride;
    prof_stride = 1;  // every pass of the tuning steps is timed
    // per variant and pass kind, the best mean pass time over the rounds; round
    // 0 (one step of each variant) only loads the kernels and warms the clocks
    double t[2][2] = {{1e30, 1e30}, {1e30, 1e30}};
    PlanTuning *pt = plan_tuning();
    PlanSlot *used[2][8] = {};
    int nused[2] = {0, 0};
    for (int round = 0; round < 3 && rc == PSS_OK; ++round)
        for (int v = 0; v < 2 && rc == PSS_OK; ++v) {
            *pt = PlanTuning{};
            pt->force = v;
            drop_graphs();
            if ((rc = profile_resolve())) break;
            profiling = true;
            for (int i = 0; i < 3; ++i) prof_ms[i] = 0, prof_n[i] = 0;
            rc = step_n(round == 0 ? 1 : k);
            if (!rc) rc = profile_resolve();
            for (int kind = 0; kind < 2 && !rc && round > 0; ++kind)
                if (prof_n[kind]) t[v][kind] = std::min(t[v][kind], prof_ms[kind] / prof_n[kind]);
            if (v == 0 && round == 0)
                for (int kind = 0; kind < 2; ++kind) {
                    nused[kind] = pt->nused[kind];
                    for (int i = 0; i < nused[kind]; ++i) used[kind][i] = pt->used[kind][i];
                }
            const int rrc = checkpoint(save, PSS_DEVICE, false);
            if (!rc) rc = rrc;
        }
    *pt = PlanTuning{};
    profiling = prof;
    prof_stride = stride;
    for (int i = 0; i < 3; ++i) prof_ms[i] = 0, prof_n[i] = 0;
    cudaFree(save);
    if (rc) return rc;
    for (int kind = 0; kind < 2; ++kind)
        for (int i = 0; i < nused[kind]; ++i) {
            const int pick = t[1][kind] < 0.98 * t[0][kind] ? 1 : 0;
            const int old = used[kind][i]->var.exchange(pick);
            if ((old < 0 ? 0 : old) != pick) ++*changed;  // an unset slot ran variant 0
        }
    if (*changed) plan_epoch().fetch_add(1);
    drop_graphs();
    graph_epoch = plan_epoch().load();
    return PSS_OK;
}

// ----------------------------------------------------------------------------
// standalone 2D transform

namespace {
std::mutex g_tw_mutex;
std::map<std::tuple<int, int, int64_t>, void *> g_tw_cache;  // (device, precision, n)

void *cached_twiddles(int dev, int precision, int64_t n, int *rc)
{
    std::lock_guard<std::mutex> lk(g_tw_mutex);
    auto key = std::make_tuple(dev, precision, n);
    auto it = g_tw_cache.find(key);
    if (it != g_tw_cache.end()) return it->second;
    void *d = nullptr;
    size_t bytes;
    std::vector<float> tf;
    std::vector<double> td;
    const void *src;
    if (precision == PSS_FP32) {
        tf = twiddles_f32(n);
        src = tf.data();
        bytes = tf.size() * 4;
    } else {
        td = twiddles_f64(n);
        src = td.data();
        bytes = td.size() * 8;
    }
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        *rc = PSS_E_OOM;
        return nullptr;
    }
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        *rc = PSS_E_CUDA;
        return nullptr;
    }
    g_tw_cache[key] = d;
    return d;
}
}  // namespace

extern "C" int pss_fft2d(void *data, int64_t nx, int64_t ny, int64_t batch, int precision, int direction,
                         void *stream)
{
    if (!data || batch < 1 || batch > 65535 || (direction != 1 && direction != -1) ||
        (precision != PSS_FP32 && precision != PSS_FP64))
        return PSS_E_ARG;
    auto ok = [](int64_t n) { return n >= 16 && n <= 8192 && (n & (n - 1)) == 0; };
    if (!ok(nx) || !ok(ny)) return PSS_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSS_E_CUDA;
    int rc = PSS_OK;
    void *twx = cached_twiddles(dev, precision, nx, &rc);
    if (!twx) return rc;
    void *twy = cached_twiddles(dev, precision, ny, &rc);
    if (!twy) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const double inv = direction > 0 ? 1.0 / (double(nx) * double(ny)) : 1.0;
    if (precision == PSS_FP32) {
        e = fft_rows<float>(static_cast<float2 *>(data), nx, batch * ny, direction, 1.0f, static_cast<float4 *>(twx), s);
        if (e == cudaSuccess)
            e = fft_cols<float>(static_cast<float2 *>(data), nx, ny, batch, direction, float(inv), static_cast<float4 *>(twy), s);
    } else {
        e = fft_rows<double>(static_cast<double2 *>(data), nx, batch * ny, direction, 1.0, static_cast<double2 *>(twx), s);
        if (e == cudaSuccess)
            e = fft_cols<double>(static_cast<double2 *>(data), nx, ny, batch, direction, inv, static_cast<double2 *>(twy), s);
    }
    return e == cudaSuccess ? PSS_OK : PSS_E_CUDA;
}
