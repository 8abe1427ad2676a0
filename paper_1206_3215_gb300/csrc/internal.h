// Internal interface between the C ABI (api.cu) and the kernel translation
// units (k_*.cu).  Launchers enqueue on the given stream and return the
// launch status; they never allocate or synchronise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pss {

template <class Rl> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <class Rl> using V2 = typename vec2<Rl>::type;

// Twiddle table entry: FP32 keeps the FP64 value as hi + lo (float4 =
// hi.re, hi.im, lo.re, lo.im) so that products are formed with one rounding
// of the exact constant; FP64 stores the value itself.
template <class Rl> struct twid;
template <> struct twid<float> { using type = float4; };
template <> struct twid<double> { using type = double2; };
template <class Rl> using TW = typename twid<Rl>::type;

// ---- plain transforms (k_fft.cu) -------------------------------------------
// dir -1 forward, +1 inverse (unnormalised); the result is multiplied by scale.
template <class Rl>
cudaError_t fft_rows(V2<Rl> *data, int64_t nx, int64_t rows_total, int dir, Rl scale,
                     const TW<Rl> *twx, cudaStream_t s);
template <class Rl>
cudaError_t fft_cols(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, int dir, Rl scale,
                     const TW<Rl> *twy, cudaStream_t s);

// ---- NLS passes (k_nls.cu) ---------------------------------------------------
// Row pass: row inverse FFT, psi <- psi exp(-i sigma dt |psi|^2), row forward FFT.
template <class Rl>
cudaError_t nls_row_pass(V2<Rl> *data, int64_t nx, int64_t rows_total, Rl sigma_dt,
                         const TW<Rl> *twx, cudaStream_t s);
// Column pass: column forward FFT, multiply by scale * a[x] * b[y]
// (a = exp(-i kx^2 tau), b = exp(-i ky^2 tau); the tables hold a - 1 and
// b - 1, stored like twiddles), column inverse FFT.
template <class Rl>
cudaError_t nls_col_pass(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, Rl scale,
                         const TW<Rl> *ax, const TW<Rl> *by, const TW<Rl> *twy, cudaStream_t s);

// ---- deterministic FP64 reductions (k_reduce.cu) -----------------------------
constexpr int RED_BLOCKS = 128;  // partial sums per field
constexpr int RED_THREADS = 256;

// NLS: per field {sum |psi|^2, sum |psi|^4} over a physical array and
// {sum |k|^2 |psi_hat|^2} over its spectrum; out[field*3 + i].
template <class Rl>
cudaError_t nls_sums(const V2<Rl> *psi, const V2<Rl> *psi_hat, int64_t nx, int64_t ny,
                     int64_t batch, const double *kx2, const double *ky2, double *partials,
                     double *out, cudaStream_t s);

// message returned by pss_last_error(NULL) for calls without a grid handle
void set_global_error(const char *msg);

// status bits written by reductions
constexpr unsigned FLAG_NONFINITE = 1u;
constexpr unsigned FLAG_NOT_CONVERGED = 2u;

}  // namespace pss
