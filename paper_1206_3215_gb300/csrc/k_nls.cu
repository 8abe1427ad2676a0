// Fused passes of the NLS split-step Fourier method (Section 4.1).
//
// The state between passes is the row transform of psi.  A row pass takes the
// row inverse transform (giving psi in physical space), applies the exact
// nonlinear sub-step psi <- exp(-i sigma |psi|^2 dt) psi and transforms the row
// forward again.  A column pass transforms the columns forward (giving
// psi_hat), applies the exact linear sub-step psi_hat <- exp(-i |k|^2 tau)
// psi_hat and transforms the columns back.  Each pass reads and writes the
// state once.
#include "launch.cuh"

namespace pss {

__device__ __forceinline__ void sincos_(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_(double a, double *s, double *c) { sincos(a, s, c); }

template <class Rl> struct NlsRow {
    V2<Rl> *data;
    Rl sigma_dt;
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void run(int64_t row, bool ok, int t, const Sm &sm,
                                        const V2<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl> v[P];
        V2<Rl> *p = data + row * N;
        load_line<P, T>(v, p, 1, t, ok);
        block_fft<N, P, +1, BLOCK>(v, sm, t, tw);
#pragma unroll
        for (int m = 0; m < P; ++m) {
            // psi exp(-i th) = psi + psi (cos th - 1 - i sin th), with
            // cos th - 1 = -2 sin^2(th/2) and sin th = 2 sin(th/2) cos(th/2):
            // no cancellation, so the modulus is kept to the final rounding.
            const Rl x = v[m].x, y = v[m].y;
            const Rl th2 = Rl(0.5) * sigma_dt * (x * x + y * y);
            Rl sh, ch;
            sincos_(th2, &sh, &ch);
            const Rl sn = Rl(2) * sh * ch, cm1 = Rl(-2) * sh * sh;
            v[m].x = x + (x * cm1 + y * sn);
            v[m].y = y + (y * cm1 - x * sn);
        }
        block_fft<N, P, -1, BLOCK>(v, sm, t, tw);
        store_line<P, T>(v, p, 1, t, ok);
    }
};

// z (h + l) with the low part only for single precision
template <bool HILO, class V> __device__ __forceinline__ V mul_hl(V z, V h, V l)
{
    if constexpr (HILO) return cadd(cmul(z, h), cmul(z, l));
    else return cmul(z, h);
}

template <class Rl> struct NlsCol {
    V2<Rl> *data;
    int64_t nx;
    Rl scale;
    const V2<Rl> *ax_hi, *ax_lo, *by_hi, *by_lo;
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void run(int64_t field, int x, int t, const Sm &sm,
                                        const V2<Rl> *tw) const
    {
        constexpr int T = N / P;
        constexpr bool HILO = sizeof(Rl) == 4;
        V2<Rl> v[P];
        V2<Rl> *p = data + field * N * nx + x;
        load_line<P, T>(v, p, nx, t, true);
        block_fft<N, P, -1, BLOCK>(v, sm, t, tw);
        const V2<Rl> ah = cscale(__ldg(ax_hi + x), scale);
        const V2<Rl> al = cscale(__ldg(ax_lo + x), scale);
#pragma unroll
        for (int m = 0; m < P; ++m) {
            const int y = t + T * m;
            V2<Rl> z = mul_hl<HILO>(v[m], ah, al);
            v[m] = mul_hl<HILO>(z, __ldg(by_hi + y), __ldg(by_lo + y));
        }
        block_fft<N, P, +1, BLOCK>(v, sm, t, tw);
        store_line<P, T>(v, p, nx, t, true);
    }
};

template <class Rl>
cudaError_t nls_row_pass(V2<Rl> *data, int64_t nx, int64_t rows_total, Rl sigma_dt,
                         const V2<Rl> *twx, cudaStream_t s)
{
    return launch_row<Rl>(nx, NlsRow<Rl>{data, sigma_dt}, twx, rows_total, s);
}

template <class Rl>
cudaError_t nls_col_pass(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, Rl scale,
                         const V2<Rl> *ax_hi, const V2<Rl> *ax_lo, const V2<Rl> *by_hi,
                         const V2<Rl> *by_lo, const V2<Rl> *twy, cudaStream_t s)
{
    return launch_col<Rl>(ny, nx, NlsCol<Rl>{data, nx, scale, ax_hi, ax_lo, by_hi, by_lo}, twy,
                          batch, s);
}

#define PSS_INST(Rl)                                                                            \
    template cudaError_t nls_row_pass<Rl>(V2<Rl> *, int64_t, int64_t, Rl, const V2<Rl> *,        \
                                          cudaStream_t);                                          \
    template cudaError_t nls_col_pass<Rl>(V2<Rl> *, int64_t, int64_t, int64_t, Rl,               \
                                          const V2<Rl> *, const V2<Rl> *, const V2<Rl> *,        \
                                          const V2<Rl> *, const V2<Rl> *, cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
