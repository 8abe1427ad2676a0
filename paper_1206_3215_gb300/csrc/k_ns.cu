// Navier-Stokes passes: loop control, row pass, derivative pass and the
// Crank-Nicolson column pass (the kernels are defined in k_ns.cuh).
#include "k_ns.cuh"

namespace pss {

// Device-side loop control, 4 ints: [0] update index k of the current pass,
// [1] any field still active after this update (built by k_ns_decide),
// [2] the value of [1] at the last k_ns_advance (read by the host loop); and
// the split column pass's item counter and epoch (FLAG_SLOT_SPLIT_CLAIM,
// FLAG_SLOT_EPOCH).
// one block per field: fold the partials of update k in a fixed order (a
// strided sum per thread, then a tree), decide, count
constexpr int NS_DECIDE_THREADS = 256;
__global__ void __launch_bounds__(NS_DECIDE_THREADS)
    k_ns_decide(NsField *fs, const double *partials, int64_t groups, int64_t batch, int *ctl, double parseval,
                double tol, int max_iter)
{
    __shared__ double red[NS_DECIDE_THREADS];
    const int64_t f = blockIdx.x;
    if (f >= batch) return;
    NsField s = fs[f];
    if (!s.active) return;  // the same for every thread of the block
    double sum = 0.0;
    for (int64_t g = threadIdx.x; g < groups; g += NS_DECIDE_THREADS) sum += partials[f * groups + g];
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int w = NS_DECIDE_THREADS / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int k = ctl[0];
    int *any_active = ctl + 1;
    const double norm = parseval * red[0];
    s.updates += 1;
    const bool done = norm < tol;
    if (done || k + 1 >= max_iter) {
        if (!done) s.nonconv = 1;
        s.idx = ns_buf(s.idx, k + 1);
        s.active = 0;
    } else {
        atomicOr(any_active, 1);
    }
    fs[f] = s;
}

__global__ void k_ns_begin(NsField *fs, int64_t batch, int *ctl)
{
    const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f == 0) {
        ctl[0] = 0;
        ctl[1] = 0;
        ctl[FLAG_SLOT_SPLIT_CLAIM] = 0;
    }
    if (f < batch) fs[f].active = 1;
}

// next update: k += 1; the loop continues while some field is active.  Inside
// a captured step graph this sets the WHILE node's condition; every field
// stops at max_iter at the latest, so the loop always ends.
__global__ void k_ns_advance(int *ctl, int use_graph, cudaGraphConditionalHandle h)
{
    const int more = ctl[1] != 0;
    ctl[2] = more;
    ctl[1] = 0;
    ctl[0] += 1;
    ctl[FLAG_SLOT_SPLIT_CLAIM] = 0;  // the next column pass claims its items from 0
    ctl[FLAG_SLOT_EPOCH] += 1;       // and publishes its tiles under a new value
    if (use_graph) cudaGraphSetConditional(h, more ? 1u : 0u);
}

template <class Rl>
cudaError_t ns_row_pass(V2<Rl> *c1, V2<Rl> *c2, const void *fs, int64_t nx, int64_t ny, int64_t batch,
                        const TW<Rl> *twx, cudaStream_t s, bool dealias, bool half)
{
    int lgy = 0;
    while ((int64_t(1) << lgy) < ny) ++lgy;  // ny is a power of two
    return launch_row<Rl>(nx, NsRow<Rl>{c1, c2, static_cast<const NsField *>(fs), lgy, dealias ? 1 : 0, half ? 1 : 0},
                          twx, batch * ny, s);
}

template <class Rl>
cudaError_t ns_col_pass(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                        const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                        const Rl *keepy, double dt, double nu, int64_t nx, int64_t ny, int64_t batch,
                        const int *ctl, int midpoint, const TW<Rl> *twy, int *groups_out, cudaStream_t s,
                        bool dealias, int64_t sx)
{
    if (sx > 0)
        return ns_col_half<Rl>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt, nu, nx, sx, ny,
                               batch, ctl, midpoint, twy, groups_out, s, dealias);
    return midpoint ? ns_col_mid<Rl>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt, nu, nx, ny,
                                     batch, ctl, twy, groups_out, s, dealias)
                    : ns_col_run<Rl, false, false>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt,
                                                   nu, nx, nx, ny, batch, ctl, twy, groups_out, s, dealias);
}

template <class Rl>
cudaError_t ns_prep_pass(V2<Rl> *const w[3], const void *fs, V2<Rl> *c1, V2<Rl> *c2, const Rl *kxo, const Rl *kyo,
                         const Rl *kx2, const Rl *ky2, int64_t nx, int64_t ny, int64_t batch,
                         const TW<Rl> *twy, cudaStream_t s, int64_t sx)
{
    if (sx > 0) return ns_prep_half<Rl>(w, fs, c1, c2, kxo, kyo, kx2, ky2, nx, sx, ny, batch, twy, s);
    NsPrep<Rl> op{w[0], w[1], w[2], static_cast<const NsField *>(fs), c1, c2, kxo, kyo, kx2, ky2,
                  Rl(1.0 / (double(nx) * double(ny))), nx, nx};
    return launch_col<Rl>(ny, nx, op, twy, batch, s);
}

cudaError_t ns_begin(void *fs, int64_t batch, int *ctl, cudaStream_t s)
{
    k_ns_begin<<<unsigned((batch + 255) / 256), 256, 0, s>>>(static_cast<NsField *>(fs), batch, ctl);
    return cudaGetLastError();
}

cudaError_t ns_decide(void *fs, const double *partials, int64_t groups, int64_t batch, int *ctl, double parseval,
                      double tol, int max_iter, cudaStream_t s)
{
    k_ns_decide<<<unsigned(batch), NS_DECIDE_THREADS, 0, s>>>(static_cast<NsField *>(fs), partials, groups,
                                                             batch, ctl, parseval, tol, max_iter);
    return cudaGetLastError();
}

cudaError_t ns_advance(int *ctl, bool use_graph, cudaGraphConditionalHandle h, cudaStream_t s)
{
    k_ns_advance<<<1, 1, 0, s>>>(ctl, use_graph ? 1 : 0, h);
    return cudaGetLastError();
}

size_t ns_field_bytes() { return sizeof(NsField); }

#define PSS_INST(Rl)                                                                                         \
    template cudaError_t ns_row_pass<Rl>(V2<Rl> *, V2<Rl> *, const void *, int64_t, int64_t, int64_t,       \
                                         const TW<Rl> *, cudaStream_t, bool, bool);                          \
    template cudaError_t ns_col_pass<Rl>(V2<Rl> *, V2<Rl> *, V2<Rl> *const[3], V2<Rl> *, void *, double *,  \
                                         const Rl *, const Rl *, const Rl *, const Rl *, const Rl *,         \
                                         const Rl *, double, double, int64_t, int64_t, int64_t,             \
                                         const int *, int, const TW<Rl> *, int *, cudaStream_t, bool,       \
                                         int64_t);                                                           \
    template cudaError_t ns_prep_pass<Rl>(V2<Rl> *const[3], const void *, V2<Rl> *, V2<Rl> *, const Rl *,     \
                                          const Rl *,                                                         \
                                          const Rl *, const Rl *, int64_t, int64_t, int64_t, const TW<Rl> *, \
                                          cudaStream_t, int64_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
