// Column pass of the implicit-midpoint Navier-Stokes variant: the Jacobian
// of (w^k + w^n)/2 in place of the trapezoidal (J^k + J^n)/2 of Section 4.3,
// with the same Crank-Nicolson diffusion (kernels in k_ns.cuh).
#include "k_ns.cuh"

namespace pss {

template <class Rl>
cudaError_t ns_col_mid(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                       const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                       const Rl *keepy, double dt, double nu, int64_t nx, int64_t ny, int64_t batch,
                       const int *ctl, const TW<Rl> *twy, int *groups_out, cudaStream_t s, bool dealias)
{
    return ns_col_run<Rl, true, false>(c1, c2, w, jn, fs, partials, kxo, kyo, kx2, ky2, keepx, keepy, dt, nu, nx,
                                       nx, ny, batch, ctl, twy, groups_out, s, dealias);
}

#define PSS_INST(Rl)                                                                                          \
    template cudaError_t ns_col_mid<Rl>(V2<Rl> *, V2<Rl> *, V2<Rl> *const[3], V2<Rl> *, void *, double *,    \
                                        const Rl *, const Rl *, const Rl *, const Rl *, const Rl *,           \
                                        const Rl *, double, double, int64_t, int64_t, int64_t, const int *,   \
                                        const TW<Rl> *, int *, cudaStream_t, bool);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
