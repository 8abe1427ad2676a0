// C ABI of the pseudospectral library: grid handles, state transfer, the
// stepping drivers of the three equations and the diagnostics.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pss.h"
#include "engine.h"

using namespace pss;

static thread_local std::string g_create_error;

void pss::set_global_error(const char *msg) { g_create_error = msg; }

// ----------------------------------------------------------------------------
// helpers

int pss_grid::fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool pow2_in_range(int64_t n) { return n >= 16 && n <= 8192 && (n & (n - 1)) == 0; }

const char *fault_env()
{
    const char *f = getenv("PSS_FAULT");
    return f ? f : "";
}

}  // namespace

// ----------------------------------------------------------------------------
// device memory of a grid

int pss_grid::alloc(void **p, size_t bytes)
{
    if (strcmp(fault_env(), "oom") == 0) return fail(PSS_E_OOM, "allocation refused (PSS_FAULT=oom)");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(PSS_E_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    owned.push_back(*p);
    return PSS_OK;
}

int pss_grid::upload(void **p, const void *host, size_t bytes)
{
    int rc = alloc(p, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(*p, host, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(PSS_E_CUDA, "table upload: %s", cudaGetErrorString(e));
    return PSS_OK;
}

int pss_grid::cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PSS_OK;
    return fail(PSS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ----------------------------------------------------------------------------
// public API

extern "C" {

void pss_default_params(pss_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->eq = PSS_EQ_NLS;
    p->precision = PSS_FP32;
    p->nx = p->ny = 64;
    p->batch = 1;
    p->x0 = p->y0 = -10.0 * M_PI;
    p->lx = p->ly = 20.0 * M_PI;
    p->dt = 1e-3;
    p->sigma = 1.0;
    p->nu = 0.1;
    p->tol = 1e-10;
    p->max_iter = 100;
    p->dealias = 1;
    p->stream = nullptr;
}

const char *pss_version(void) { return "pss 0.1 (sm_103a)"; }

const char *pss_last_error(const pss_grid *g)
{
    if (!g) return g_create_error.c_str();
    return g->err.c_str();
}

int pss_create_grid(pss_grid **out, const pss_params *p)
{
    if (!out || !p) {
        g_create_error = "null argument";
        return PSS_E_ARG;
    }
    *out = nullptr;
    const char *bad = nullptr;
    if (p->eq < PSS_EQ_NLS || p->eq > PSS_EQ_NS) bad = "eq";
    else if (p->precision != PSS_FP32 && p->precision != PSS_FP64) bad = "precision";
    else if (!pow2_in_range(p->nx) || !pow2_in_range(p->ny)) bad = "nx/ny (powers of two in [16, 8192])";
    else if (p->batch < 1 || p->batch > 65535) bad = "batch (1..65535)";
    else if (!(p->lx > 0) || !(p->ly > 0) || !std::isfinite(p->lx) || !std::isfinite(p->ly)) bad = "lx/ly";
    else if (!(p->dt > 0) || !std::isfinite(p->dt)) bad = "dt";
    else if (!std::isfinite(p->sigma)) bad = "sigma";
    else if (p->eq == PSS_EQ_NS && (!(p->nu >= 0) || !(p->tol > 0) || p->max_iter < 1)) bad = "nu/tol/max_iter";
    else if (p->scheme != PSS_NS_CN && p->scheme != PSS_NS_MIDPOINT) bad = "scheme";
    else if (p->rfft != 0 && p->rfft != 1) bad = "rfft (0 or 1)";
    else if (p->rfft && p->eq == PSS_EQ_NLS) bad = "rfft (sine-Gordon and Navier-Stokes only)";
    if (bad) {
        g_create_error = std::string("invalid parameter: ") + bad;
        return PSS_E_ARG;
    }
    pss_grid *g = new pss_grid();
    g->p = *p;
    if (strcmp(fault_env(), "nonconv") == 0) g->p.max_iter = 1;
    int rc = g->init();
    if (rc) {
        g_create_error = g->err;
        pss_destroy(g);
        return rc;
    }
    *out = g;
    return PSS_OK;
}

int pss_destroy(pss_grid *g)
{
    if (!g) return PSS_OK;
    {
        DeviceGuard dg(g->dev);
        if (g->stream) cudaStreamSynchronize(g->stream);
        for (void *q : g->owned) cudaFree(q);
        for (void *q : g->owned_host) cudaFreeHost(q);
        g->release_extra();
        if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    }
    delete g;
    return PSS_OK;
}

int pss_set_state(pss_grid *g, const void *a, const void *b, int where)
{
    if (!g) return PSS_E_ARG;
    if (!a || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "set_state: null state or bad location");
    DeviceGuard dg(g->dev);
    return g->set_state(a, b, where);
}

int pss_step_n(pss_grid *g, int64_t n)
{
    if (!g) return PSS_E_ARG;
    if (n < 0) return g->fail(PSS_E_ARG, "step_n: n < 0");
    if (!g->has_state) return g->fail(PSS_E_STATE, "step_n before set_state");
    DeviceGuard dg(g->dev);
    return g->step_n(n);
}

int pss_set_state_sg_levels(pss_grid *g, const void *u_n, const void *u_nm1, int where)
{
    if (!g) return PSS_E_ARG;
    if (g->p.eq != PSS_EQ_SG) return g->fail(PSS_E_ARG, "set_state_sg_levels: not a sine-Gordon grid");
    if (!u_n || !u_nm1 || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "set_state_sg_levels: null buffer or bad location");
    DeviceGuard dg(g->dev);
    return g->set_sg_levels(u_n, u_nm1, where);
}

int pss_step_n_batch(pss_grid *const *grids, int count, const int64_t *n)
{
    if (count < 0 || (count > 0 && (!grids || !n))) return PSS_E_ARG;
    for (int i = 0; i < count; ++i)
        if (!grids[i]) return PSS_E_ARG;
    int first = PSS_OK;
    for (int i = 0; i < count; ++i) {
        const int rc = pss_step_n(grids[i], n[i]);
        if (rc != PSS_OK && first == PSS_OK) first = rc;
    }
    return first;
}

int pss_autotune(pss_grid *g, int steps, int *changed)
{
    if (!g) return PSS_E_ARG;
    if (!changed || steps < 1) return g->fail(PSS_E_ARG, "autotune: steps < 1 or null output");
    DeviceGuard dg(g->dev);
    return g->autotune(steps, changed);
}

int pss_get_state(pss_grid *g, void *a, void *b, int where)
{
    if (!g) return PSS_E_ARG;
    if (!a || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "get_state: null buffer or bad location");
    if (!g->has_state) return g->fail(PSS_E_STATE, "get_state before set_state");
    DeviceGuard dg(g->dev);
    return g->get_state(a, b, where);
}

int pss_set_field(pss_grid *g, int64_t field, const void *a, const void *b, int where)
{
    if (!g) return PSS_E_ARG;
    if (!a || field < 0 || field >= g->batch || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "set_field: bad field, pointer or location");
    DeviceGuard dg(g->dev);
    return g->set_field(field, a, b, where);
}

int pss_get_field(pss_grid *g, int64_t field, void *a, void *b, int where)
{
    if (!g) return PSS_E_ARG;
    if (!a || field < 0 || field >= g->batch || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "get_field: bad field, pointer or location");
    if (!g->has_state) return g->fail(PSS_E_STATE, "get_field before any state was set");
    DeviceGuard dg(g->dev);
    return g->get_field(field, a, b, where);
}

int pss_conserved_quantities(pss_grid *g, double *out, int cap, int *count)
{
    if (!g) return PSS_E_ARG;
    if (!out || !count) return g->fail(PSS_E_ARG, "conserved_quantities: null pointer");
    if (!g->has_state) return g->fail(PSS_E_STATE, "conserved_quantities before set_state");
    const int per = g->p.eq == PSS_EQ_NLS ? 2 : g->p.eq == PSS_EQ_SG ? 1 : 3;
    const int64_t need = per * g->p.batch;
    *count = int(need);
    if (cap < need) return g->fail(PSS_E_ARG, "conserved_quantities: cap %d < %lld", cap, (long long)need);
    DeviceGuard dg(g->dev);
    return g->conserved(out);
}

int pss_stats(pss_grid *g, int64_t *steps, int64_t *ns_updates)
{
    if (!g) return PSS_E_ARG;
    DeviceGuard dg(g->dev);
    int rc = g->sync();
    if (steps) *steps = g->steps;
    if (ns_updates) {
        int r2 = g->ns_update_count(ns_updates);
        if (!rc) rc = r2;
    }
    return rc;
}

int pss_set_profiling(pss_grid *g, int on)
{
    if (!g) return PSS_E_ARG;
    DeviceGuard dg(g->dev);
    int rc = g->profile_resolve();
    if (rc) return rc;
    if (on < 0) return g->fail(PSS_E_ARG, "set_profiling: on must be >= 0");
    g->profiling = on != 0;
    g->prof_stride = on > 1 ? on : 1;
    for (int k = 0; k < 3; ++k) {
        g->prof_ms[k] = 0;
        g->prof_n[k] = 0;
    }
    g->launches = 0;
    return PSS_OK;
}

int pss_profile_read(pss_grid *g, double *out, int cap, int *count)
{
    if (!g) return PSS_E_ARG;
    if (!out || !count) return g->fail(PSS_E_ARG, "profile_read: null pointer");
    *count = 7;
    if (cap < 7) return g->fail(PSS_E_ARG, "profile_read: cap < 7");
    DeviceGuard dg(g->dev);
    int rc = g->profile_resolve();
    if (rc) return rc;
    out[0] = double(g->launches);
    for (int k = 0; k < 3; ++k) {
        out[1 + 2 * k] = double(g->prof_n[k]);
        out[2 + 2 * k] = g->prof_ms[k];
    }
    return PSS_OK;
}

int pss_sync(pss_grid *g)
{
    if (!g) return PSS_E_ARG;
    DeviceGuard dg(g->dev);
    return g->sync();
}

int pss_checkpoint_size(const pss_grid *g, size_t *bytes)
{
    if (!g || !bytes) return PSS_E_ARG;
    *bytes = g->checkpoint_bytes();
    return PSS_OK;
}

int pss_checkpoint_save(pss_grid *g, void *buf, int where)
{
    if (!g) return PSS_E_ARG;
    if (!buf || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "checkpoint_save: bad buffer");
    if (!g->has_state) return g->fail(PSS_E_STATE, "checkpoint_save before set_state");
    DeviceGuard dg(g->dev);
    return g->checkpoint(buf, where, true);
}

int pss_checkpoint_load(pss_grid *g, const void *buf, int where)
{
    if (!g) return PSS_E_ARG;
    if (!buf || (where != PSS_HOST && where != PSS_DEVICE))
        return g->fail(PSS_E_ARG, "checkpoint_load: bad buffer");
    DeviceGuard dg(g->dev);
    return g->checkpoint(const_cast<void *>(buf), where, false);
}

}  // extern "C"
