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
// b - 1, stored like twiddles), column inverse FFT.  *status gets
// STATUS_TMA_TIMEOUT if a tile copy never arrived (the pass is then incomplete).
template <class Rl>
cudaError_t nls_col_pass(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, Rl scale,
                         const TW<Rl> *ax, const TW<Rl> *by, const TW<Rl> *twy, int *status, cudaStream_t s);

// ---- sine-Gordon passes (k_sg.cu) ---------------------------------------------
// Row pass on H (column inverse transform of uhat^n / (nx ny)): row inverse
// FFT, s = sin(Re), row forward FFT, in place.
template <class Rl>
cudaError_t sg_row_pass(V2<Rl> *h, int64_t nx, int64_t rows_total, const TW<Rl> *twx, cudaStream_t s);
// Column pass: column FFT of S = F sin u^n; d <- d - (a u + dt^2 S)/(1 + a/4),
// u <- u + d (a = dt^2 |k|^2), in place; H <- column inverse FFT of u / (nreal ny).
// nx is the row stride (columns processed), nreal the real row length (0: nx).
// *status gets STATUS_TMA_TIMEOUT if a tile copy never arrived.
template <class Rl>
cudaError_t sg_col_pass(V2<Rl> *h, V2<Rl> *u, V2<Rl> *d, int64_t nx, int64_t ny, int64_t batch,
                        const Rl *kx2, const Rl *ky2, Rl dt, const TW<Rl> *twy, int *status, cudaStream_t s,
                        int64_t nreal = 0);
// Half-spectrum (real-to-complex) sine-Gordon row pass, k_sg_r2c.cu: rows of
// stride sx holding kx = 0 .. nx/2; twm: twiddles of length nx/2, twn: of nx.
template <class Rl>
cudaError_t sg_row_pass_r2c(V2<Rl> *h, int64_t nx, int64_t sx, int64_t rows_total, const TW<Rl> *twm,
                            const TW<Rl> *twn, cudaStream_t s);
// full [batch][ny][nx] spectrum of real fields <-> half spectrum [batch][ny][sx]
template <class Rl>
cudaError_t pack_half(const V2<Rl> *full, V2<Rl> *half, int64_t nx, int64_t ny, int64_t sx, int64_t batch,
                      cudaStream_t s);
template <class Rl>
cudaError_t unpack_half(const V2<Rl> *half, V2<Rl> *full, int64_t nx, int64_t ny, int64_t sx, int64_t batch,
                        cudaStream_t s);

// ---- Navier-Stokes passes (k_ns.cu) -------------------------------------------
size_t ns_field_bytes();  // bytes of the per-field fixed-point record
template <class Rl>
cudaError_t ns_row_pass(V2<Rl> *c1, V2<Rl> *c2, const void *fs, int64_t nx, int64_t ny, int64_t batch,
                        const TW<Rl> *twx, cudaStream_t s, bool dealias, bool half = false);
template <class Rl>
cudaError_t ns_col_pass(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                        const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                        const Rl *keepy, double dt, double nu, int64_t nx, int64_t ny, int64_t batch,
                        const int *ctl, int midpoint, const TW<Rl> *twy, int *groups_out, cudaStream_t s,
                        bool dealias, int64_t sx = 0);
template <class Rl>
cudaError_t ns_prep_pass(V2<Rl> *const w[3], const void *fs, V2<Rl> *c1, V2<Rl> *c2, const Rl *kxo, const Rl *kyo,
                         const Rl *kx2, const Rl *ky2, int64_t nx, int64_t ny, int64_t batch,
                         const TW<Rl> *twy, cudaStream_t s, int64_t sx = 0);
// loop control ctl (4 ints on the device): [0] update index, [1] any field
// active after the current update, [2] its value at the last advance
cudaError_t ns_begin(void *fs, int64_t batch, int *ctl, cudaStream_t s);
cudaError_t ns_decide(void *fs, const double *partials, int64_t groups, int64_t batch, int *ctl, double parseval,
                      double tol, int max_iter, cudaStream_t s);
cudaError_t ns_advance(int *ctl, bool use_graph, cudaGraphConditionalHandle h, cudaStream_t s);

// ---- elementwise helpers (k_util.cu) ----------------------------------------
template <class Rl> cudaError_t real_to_complex(const Rl *src, V2<Rl> *dst, int64_t n, bool apply_sin, cudaStream_t s);
template <class Rl>
cudaError_t complex_to_real(const V2<Rl> *a, const V2<Rl> *b, Rl c, Rl *dst, int64_t n, cudaStream_t s);
template <class Rl>
cudaError_t sg_init(const V2<Rl> *u, V2<Rl> *d, const V2<Rl> *sn, const double *kx2, const double *ky2, double dt,
                    int64_t nx, int64_t ny, int64_t batch, cudaStream_t s);
template <class Rl>
cudaError_t ns_gather(const void *fs, V2<Rl> *const w[3], V2<Rl> *dst, int64_t per_field, int64_t batch,
                      cudaStream_t s);
template <class Rl> cudaError_t cplx_axpy(const V2<Rl> *a, const V2<Rl> *b, Rl c, V2<Rl> *dst, int64_t n, cudaStream_t s);
template <class Rl>
cudaError_t apply_mask(V2<Rl> *a, const Rl *keepx, const Rl *keepy, int64_t nx, int64_t ny, int64_t batch, cudaStream_t s);

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

// SG: per field {sum (Y/dt)^2/2, sum 1 - cos(X - Y/2), sum |k|^2 |U - D/2|^2}
template <class Rl>
cudaError_t sg_sums(const V2<Rl> *X, const V2<Rl> *Y, const V2<Rl> *U, const V2<Rl> *D, int64_t nx, int64_t ny,
                    int64_t batch, const double *kx2, const double *ky2, double dt, double *partials, double *out,
                    cudaStream_t s);
// NS: per field {Re w_hat(0,0), sum |w_hat|^2, sum_{k != 0} |w_hat|^2 / |k|^2}
template <class Rl>
cudaError_t ns_sums(const void *fs, V2<Rl> *const w[3], int64_t nx, int64_t ny, int64_t batch, const double *kx2,
                    const double *ky2, double *partials, double *out, cudaStream_t s);

// status bits written by reductions
constexpr unsigned FLAG_NONFINITE = 1u;
constexpr unsigned FLAG_NOT_CONVERGED = 2u;

// int slot of the grid's 64-byte device flag block that pass kernels report
// a lost tile copy in (slots 0 .. 3 carry the NS step control)
constexpr int FLAG_SLOT_PASS_STATUS = 8;
// NS split column pass: slot 4 its item counter (zeroed by k_ns_begin and
// k_ns_advance), slot 5 the column-pass epoch (never reset; k_ns_advance
// adds one), and from int FLAG_TILE_DONE on one word per column tile
// (batch x nx words, allocated after the 64-byte block for NS grids)
constexpr int FLAG_SLOT_SPLIT_CLAIM = 4;
constexpr int FLAG_SLOT_EPOCH = 5;
constexpr int FLAG_TILE_DONE = 16;

}  // namespace pss
