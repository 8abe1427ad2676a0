// Navier-Stokes passes on half spectra (kx = 0 .. nx/2, real-to-complex in
// x): the column pass for both schemes and the derivative pass (kernels in
// k_ns.cuh).  The vorticity iterates and J_hat^n hold half the columns; the
// derivative fields C1, C2 the row pass transforms stay full width and are
// written at kx and nx - kx from each visited column.
#include "k_ns.cuh"

namespace pss {

template <class Rl>
cudaError_t ns_col_half(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                        const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                        const Rl *keepy, double dt, double nu, int64_t nxf, int64_t sx, int64_t ny, int64_t batch,
                        const int *ctl, int midpoint, const TW<Rl> *twy, int *groups_out, cudaStream_t s,
                        bool dealias)
{
    if (midpoint)
        return ns_col_run<Rl, true, true>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt, nu, nxf,
                                          sx, ny, batch, ctl, twy, groups_out, s, dealias);
    return ns_col_run<Rl, false, true>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt, nu, nxf,
                                       sx, ny, batch, ctl, twy, groups_out, s, dealias);
}

template <class Rl>
cudaError_t ns_prep_half(V2<Rl> *const w[3], const void *fs, V2<Rl> *c1, V2<Rl> *c2, const Rl *kxo, const Rl *kyo,
                         const Rl *kx2, const Rl *ky2, int64_t nxf, int64_t sx, int64_t ny, int64_t batch,
                         const TW<Rl> *twy, cudaStream_t s)
{
    NsPrep<Rl, true> op{w[0], w[1], w[2], static_cast<const NsField *>(fs), c1, c2, kxo, kyo, kx2, ky2,
                        Rl(1.0 / (double(nxf) * double(ny))), sx, nxf};
    return launch_col<Rl>(ny, sx, op, twy, batch, s);
}

#define PSS_INST(Rl)                                                                                         \
    template cudaError_t ns_col_half<Rl>(V2<Rl> *, V2<Rl> *, V2<Rl> *const[3], V2<Rl> *, void *, double *,  \
                                         const Rl *, const Rl *, const Rl *, const Rl *, const Rl *,         \
                                         const Rl *, double, double, int64_t, int64_t, int64_t, int64_t,    \
                                         const int *, int, const TW<Rl> *, int *, cudaStream_t, bool);      \
    template cudaError_t ns_prep_half<Rl>(V2<Rl> *const[3], const void *, V2<Rl> *, V2<Rl> *, const Rl *,     \
                                          const Rl *, const Rl *, const Rl *, int64_t, int64_t, int64_t,     \
                                          int64_t, const TW<Rl> *, cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
