// The grid handle behind the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pss.h"
#include "internal.h"

struct pss_grid {
    pss_params p{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t nx = 0, ny = 0, batch = 0, npts = 0, ntot = 0;
    size_t esz = 0;  // bytes of one complex element
    std::string err;

    std::vector<void *> owned;       // cudaMalloc'd, freed by pss_destroy
    std::vector<void *> owned_host;  // cudaMallocHost'd

    // complex work arrays, ntot elements each (meaning depends on eq)
    void *buf[8] = {};
    int nbuf = 0;

    // sine-Gordon on half spectra (p.rfft): the stepping state lives in
    // hbuf = {uhat, d, H}, [batch][ny][sx] with kx = 0 .. nx/2; the full
    // buffers buf[0], buf[1] are rebuilt from it when a call reads the state
    bool half = false;
    int64_t sx = 0;
    void *hbuf[3] = {};
    void *twm = nullptr;   // twiddles of length nx/2
    void *kx2h = nullptr;  // kx^2 of the half-spectrum columns (0 beyond nx/2)
    bool half_valid = false, full_valid = true;
    int half_sync(bool to_half);  // make the half (true) or full (false) copy current
    // Navier-Stokes on half spectra (p.rfft): the vorticity iterates and
    // J_hat^n in buf[0..3] hold [batch][ny][nsx] (kx = 0 .. nx/2); C1, C2 and
    // the scratch buf[6] stay full width
    bool ns_half = false;
    int64_t nsx = 0;

    // tables (device)
    void *twx = nullptr, *twy = nullptr;                           // twiddles, precision
    void *ax[2] = {}, *by[2] = {};  // NLS exp(-i k^2 tau) per axis, [dt/2, dt]
    double *kx2d = nullptr, *ky2d = nullptr;                       // |k|^2 per axis, FP64
    void *kx2 = nullptr, *ky2 = nullptr;                           // |k|^2 per axis, precision
    void *kxo = nullptr, *kyo = nullptr;                           // odd-derivative k, precision
    void *keepx = nullptr, *keepy = nullptr;                       // NS dealias mask (0/1), precision

    // reductions
    double *partials = nullptr;  // batch * RED_BLOCKS * 3 (and NS per-tile partials)
    double *sums = nullptr;      // batch * 3
    double *host_sums = nullptr; // pinned, batch * 3
    unsigned *flags = nullptr;   // device status bits
    unsigned *host_flags = nullptr;

    // NS fixed-point bookkeeping (device, per field)
    void *ns_field = nullptr;     // device, batch records (see k_ns.cu)
    void *host_fields = nullptr;  // pinned copy of the records

    // tracing: event pairs around passes (kind 0 row, 1 column, 2 other);
    // with prof_stride S > 1 only the passes of every S-th step are timed
    // (pass pairs 0, S, 2S, ... of a pss_step_n call)
    bool profiling = false;
    int prof_stride = 1;
    int64_t prof_pass = 0;   // passes seen in the current pss_step_n call
    bool prof_open = false;  // the pass being run is timed
    bool sampled(int64_t pass) const { return prof_stride <= 1 || (pass / 2) % prof_stride == 0; }
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;  // kind of pair i = events 2i, 2i+1
    double prof_ms[3] = {0, 0, 0};
    int64_t prof_n[3] = {0, 0, 0};
    int64_t launches = 0;
    int pass_begin(int kind);
    int pass_end();
    int profile_resolve();

    // captured CUDA graphs (NLS/SG: also while profiling; NS: off while
    // profiling; all off with PSS_GRAPHS=0)
    bool use_graphs = true;
    cudaGraph_t ns_graph = nullptr;       // one NS step: begin -> WHILE(active) { passes }
    cudaGraphExec_t ns_exec = nullptr;
    cudaGraphConditionalHandle ns_cond = 0;
    // NLS/SG step_n(n) as one graph, by (n, profiling stride).  A profiling
    // graph records an event pair around each timed pass (its own events)
    // and the kind of each timed pass.
    struct StepGraph {
        int64_t n = 0;
        int prof = 0;  // 0: no events; else the profiling stride
        cudaGraphExec_t exec = nullptr;
        int64_t passes = 0;
        std::vector<cudaEvent_t> evs;
        std::vector<int> kinds;
    };
    std::vector<StepGraph> step_graphs;
    const StepGraph *prof_pending = nullptr;  // profiling graph launched, not yet read
    StepGraph *capturing = nullptr;           // profiling graph being captured
    int graph_epoch = 0;  // plan epoch the cached graphs were captured under
    static void free_step_graph(StepGraph &g)
    {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t e : g.evs) cudaEventDestroy(e);
        g.exec = nullptr;
        g.evs.clear();
    }
    void drop_graphs()
    {
        if (ns_exec) cudaGraphExecDestroy(ns_exec);
        if (ns_graph) cudaGraphDestroy(ns_graph);
        if (prof_pending) cudaStreamSynchronize(stream);  // its events must not be destroyed in flight
        prof_pending = nullptr;
        for (auto &g : step_graphs) free_step_graph(g);
        step_graphs.clear();
        ns_exec = nullptr;
        ns_graph = nullptr;
    }
    int autotune(int steps, int *changed);

    int64_t steps = 0;
    bool has_state = false;
    bool nonconv_pending = false;

    int fail(int code, const char *fmt, ...);
    int alloc(void **p, size_t bytes);
    int upload(void **p, const void *host, size_t bytes);
    int cuda(cudaError_t e, const char *what);

    int init();
    int set_state(const void *a, const void *b, int where);
    int set_sg_levels(const void *u_n, const void *u_nm1, int where);
    int step_n(int64_t n);
    int get_state(void *a, void *b, int where);
    int set_field(int64_t f, const void *a, const void *b, int where);
    int get_field(int64_t f, void *a, void *b, int where);
    int conserved(double *out);
    int sync();
    int ns_update_count(int64_t *n);
    size_t checkpoint_bytes() const;
    int checkpoint(void *buf, int where, bool save);
    void release_extra()
    {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        ev_pool.clear();
        drop_graphs();
    }
    int check_ns_nonconv();
    int check_pass_status();

    size_t field_bytes() const { return size_t(ntot) * esz; }
    double dA() const { return (p.lx / double(nx)) * (p.ly / double(ny)); }
};
