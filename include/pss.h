/*
 * pss — Fourier pseudospectral time stepping on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library.  It advances the three periodic 2D equations of
 * Cloutier, Muite and Rigge, "Performance of FORTRAN and C GPU Extensions for
 * a Benchmark Suite of Fourier Pseudospectral Algorithms" (arXiv:1206.3215):
 *
 *   NLS  i psi_t + psi_xx + psi_yy = sigma |psi|^2 psi          (Eq. 1)
 *        Strang split-step Fourier                               (Section 4.1)
 *   SG   u_tt - Lap u = -sin u                                   (Eq. 3)
 *        semi-implicit leapfrog, Lap averaged over n+1, n, n-1   (Section 4.2)
 *   NS   omega_t + psi_y omega_x - psi_x omega_y = nu Lap omega,
 *        Lap psi = -omega                                         (Section 3.3)
 *        Crank-Nicolson with fixed-point iteration on the
 *        Jacobian                                                 (Section 4.3)
 *
 * Every transform is the library's own hand-written Stockham FFT; the
 * pointwise nonlinearity is fused into the row pass and the k-space operator
 * into the column pass, so one time step is two passes over the state.
 *
 * Conventions
 *  - Grids are nx * ny points, both powers of two in [16, 8192], on the box
 *    [x0, x0+lx) x [y0, y0+ly); x_j = x0 + j lx / nx.  Arrays are row-major
 *    [batch][ny][nx] with x fastest.  Complex values are interleaved (re, im).
 *  - Wavenumbers are k = 2 pi m / L, m in {0, .., n/2-1, -n/2, .., -1};
 *    |k|^2 includes the Nyquist mode m = -n/2.
 *  - Precision PSS_FP32 stores and computes in float (complex64 state),
 *    PSS_FP64 in double.  Twiddle and propagator tables are computed on the
 *    host in double and rounded once.  Conserved quantities are accumulated
 *    in double on the device in a fixed order.
 *  - Every call returns a status code (PSS_OK = 0).  After an error,
 *    pss_last_error() describes it; the handle stays valid and may be
 *    destroyed.  A handle is not thread safe: use one per host thread.
 *  - The library owns all device memory of a grid (allocated by
 *    pss_create_grid, freed by pss_destroy); the caller owns host buffers and
 *    any device buffer it passes in.
 *  - Work is enqueued on the grid's stream (params.stream, or a stream the
 *    library creates when it is NULL).  pss_step_n is asynchronous;
 *    pss_get_state, pss_conserved_quantities and pss_sync synchronise.
 */
#ifndef PSS_H
#define PSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PSS_OK 0
#define PSS_E_ARG 1           /* invalid argument (size, pointer, enum, range)       */
#define PSS_E_OOM 2           /* device or host allocation failed                    */
#define PSS_E_CUDA 3          /* a CUDA runtime call failed                          */
#define PSS_E_NOT_CONVERGED 4 /* NS fixed point reached max_iter in some step        */
#define PSS_E_NONFINITE 5     /* a NaN or Inf appeared in a reduction                */
#define PSS_E_STATE 6         /* call out of order (e.g. step before set_state)      */

/* equations */
#define PSS_EQ_NLS 0
#define PSS_EQ_SG 1
#define PSS_EQ_NS 2

/* precisions */
#define PSS_FP32 0
#define PSS_FP64 1

/* Navier-Stokes time discretisations (pss_params.scheme) */
#define PSS_NS_CN 0       /* Crank-Nicolson diffusion, trapezoidal Jacobian (J^k + J^n)/2,
                             Section 4.3 (the default)                                   */
#define PSS_NS_MIDPOINT 1 /* same diffusion, Jacobian of the midpoint (w^k + w^n)/2:
                             the implicit midpoint rule, which keeps energy and
                             enstrophy of the dealiased inviscid system exactly          */

/* location of a caller buffer */
#define PSS_HOST 0
#define PSS_DEVICE 1

typedef struct pss_params {
    int32_t eq;        /* PSS_EQ_NLS / PSS_EQ_SG / PSS_EQ_NS                           */
    int32_t precision; /* PSS_FP32 / PSS_FP64                                          */
    int64_t nx, ny;    /* grid points, powers of two in [16, 8192]                     */
    int64_t batch;     /* independent fields advanced together, >= 1                   */
    double x0, y0;     /* box origin (only used by callers to place initial data)      */
    double lx, ly;     /* box lengths, > 0                                             */
    double dt;         /* time step, > 0                                               */
    double sigma;      /* NLS: coefficient of |psi|^2 psi (Eq. 1 has +1)               */
    double nu;         /* NS: viscosity (the paper's Taylor-Green runs use 1/10)       */
    double tol;        /* NS: fixed-point tolerance on integral (dw)^2 (paper: 1e-10)  */
    int32_t max_iter;  /* NS: bound on fixed-point updates per step (default 100)     */
    int32_t dealias;   /* NS: 1 = 2/3-rule square truncation (3|m| < n) on J and w0   */
    void *stream;      /* cudaStream_t to enqueue on, or NULL for a library stream    */
    int32_t scheme;    /* NS: PSS_NS_CN or PSS_NS_MIDPOINT                             */
    int32_t rfft;      /* SG, NS: 1 = keep the k-space state as half spectra
                          (kx = 0 .. nx/2, the real fields' other half being its
                          conjugate; the paper's programs used real-to-complex
                          transforms for both, Sections 5.2-5.3); 0 = full complex
                          spectra.  Must be 0 for NLS.                             */
} pss_params;

typedef struct pss_grid pss_grid;

/* Fill *p with defaults: NLS, FP32, 64x64, batch 1, box [-10pi,10pi)^2,
 * dt 1e-3, sigma +1, nu 1/10, tol 1e-10, max_iter 100, dealias 1,
 * scheme PSS_NS_CN, rfft 0. */
void pss_default_params(pss_params *p);

/* Create a grid: validates *p, allocates every device buffer the equation
 * needs (no allocation happens later on the stepping path), and uploads the
 * FP64-generated twiddle and wavenumber tables.
 * Errors: PSS_E_ARG (bad field; *out = NULL), PSS_E_OOM, PSS_E_CUDA. */
int pss_create_grid(pss_grid **out, const pss_params *p);

/* Set the initial state; resets the step counter and the NS iteration count.
 *  NLS: a = psi, interleaved complex [batch][ny][nx]; b unused (may be NULL).
 *  SG:  a = u(0), b = u_t(0), real [batch][ny][nx] (b NULL means u_t(0) = 0).
 *       u^{-1} is formed by the second-order backward Taylor step
 *       u^{-1} = u^0 - dt u_t(0) + dt^2/2 (Lap u^0 - sin u^0)   (Section 4.2 start-up).
 *  NS:  a = omega(0), real [batch][ny][nx]; masked by the 2/3 rule if dealias.
 * Element type follows the precision (float or double).  where = PSS_HOST or
 * PSS_DEVICE; device buffers must be on the grid's device.  Synchronises the
 * grid's stream before returning when where = PSS_HOST. */
int pss_set_state(pss_grid *g, const void *a, const void *b, int where);

/* Advance every field of the batch by n >= 0 time steps, enqueued on the grid
 * stream.  NLS: L(dt/2) N(dt) L(dt/2) per step (Section 4.1), executed as
 * L(dt/2) [N L(dt)]^(n-1) N L(dt/2).  SG: Section 4.2.  NS: Section 4.3; if a
 * step reaches max_iter the iterate at max_iter is accepted and
 * PSS_E_NOT_CONVERGED is returned by this call or by the next synchronising
 * call.  Errors: PSS_E_STATE (no state set), PSS_E_ARG (n < 0). */
int pss_step_n(pss_grid *g, int64_t n);

/* Sine-Gordon: set both time levels from u^n (a) and u^{n-1} (b), real
 * [batch][ny][nx] in the grid's precision, instead of the start-up from
 * u(0), u_t(0) of pss_set_state: uhat^n = F u^n, uhat^{n-1} = F u^{n-1}
 * (e.g. to continue from two levels read back by pss_get_state; the exact
 * bitwise resume is pss_checkpoint_*).  Resets the step counter.
 * Errors: PSS_E_ARG (not a sine-Gordon grid, null pointer, bad location). */
int pss_set_state_sg_levels(pss_grid *g, const void *u_n, const void *u_nm1, int where);

/* Advance several grids in one call: grids[i] by n[i] >= 0 steps, each
 * enqueued on its own grid's stream (grids on different streams run
 * concurrently on the device).  Every grid is attempted; the return value is
 * the first error, with that grid's message in pss_last_error(grids[i]).
 * Errors: PSS_E_ARG (count < 0, null arrays or a null grid). */
int pss_step_n_batch(pss_grid *const *grids, int count, const int64_t *n);

/* Autotuner (plans).  The FP32 row and column pass kernels of length >= 512
 * are compiled in two launch shapes: 32 points per thread with two CTAs per
 * SM, and 16 points per thread with four.  pss_autotune times `steps` steps
 * of this grid in each (on its current state, which is restored afterwards,
 * step counter included) and records, per pass kernel, the faster one in a
 * process-wide plan keyed by (equation, grid size, precision): every grid of
 * that key then runs the same kernels, so batched and single runs stay equal.
 * The shapes round differently (different transform factorisations), so a
 * plan change alters results at the rounding level; cached step graphs are
 * re-captured.  *changed receives the number of kernels whose plan changed.
 * NLS and sine-Gordon FP32 grids only (others return 0 changes).  Setting the
 * environment variable PSS_PLAN=0 or 1 pins every kernel to one shape.
 * Errors: PSS_E_STATE (no state), PSS_E_OOM (no room for the state copy). */
int pss_autotune(pss_grid *g, int steps, int *changed);

/* Copy the state back (inverse of pss_set_state's layout).
 *  NLS: a = psi (complex).  SG: a = u^n, b = u^{n-1} (real; b may be NULL).
 *  NS:  a = omega^n (real).  Synchronises. */
int pss_get_state(pss_grid *g, void *a, void *b, int where);

/* One field of the batch (a slot), for callers that manage fields
 * independently (continuous batching): the same layouts as pss_set_state /
 * pss_get_state for a single [ny][nx] field, with the same set-up of the
 * equation's state for that field only; the other fields are untouched.
 * pss_set_field does not change the grid's step counter.  Work is enqueued on
 * the grid's stream; pss_set_field synchronises for HOST input,
 * pss_get_field always.  Fields never set hold zeros (a fixed point of all
 * three equations).  Errors: PSS_E_ARG (field out of range, null pointer). */
int pss_set_field(pss_grid *g, int64_t field, const void *a, const void *b, int where);
int pss_get_field(pss_grid *g, int64_t field, void *a, void *b, int where);

/* Diagnostics of every field, in double, written to out[field * per + i]:
 *  NLS (per = 2): mass  = integral |psi|^2,
 *                 energy = integral |grad psi|^2 / 2 + sigma |psi|^4 / 4   (Eq. 2);
 *  SG  (per = 1): H at t_{n-1/2}: integral (u^n-u^{n-1})^2/(2dt^2) + 1 - cos(ubar)
 *                 + |grad ubar|^2 / 2, ubar = (u^n+u^{n-1})/2            (Section 3.2);
 *  NS  (per = 3): integral omega, integral omega^2 / 2, integral |u|^2 / 2.
 * cap is the capacity of out in doubles; *count receives batch * per.
 * Synchronises.  PSS_E_ARG if cap is too small; PSS_E_NONFINITE if a sum is
 * not finite (values are still written). */
int pss_conserved_quantities(pss_grid *g, double *out, int cap, int *count);

/* Steps taken since set_state, and (NS) total fixed-point updates
 * (= Jacobian evaluations) summed over steps and fields.  Synchronises. */
int pss_stats(pss_grid *g, int64_t *steps, int64_t *ns_updates);

/* Checkpoint of the exact internal state (bitwise resume).
 * pss_checkpoint_size gives the byte count; save/load copy to or from a
 * caller buffer at `where`.  Loading restores the step counter too. */
int pss_checkpoint_size(const pss_grid *g, size_t *bytes);
int pss_checkpoint_save(pss_grid *g, void *buf, int where);
int pss_checkpoint_load(pss_grid *g, const void *buf, int where);

/* Pass timing (tracing).  on = 0: off (the default); on = 1: pss_step_n
 * records a CUDA event pair around every row pass and every column pass on
 * the grid's stream; on = S > 1: only around the passes of every S-th step
 * (pass pairs 0, S, 2S, ... of each pss_step_n call), which leaves the
 * stepping speed as it is (an event pair costs a few microseconds per pass).
 * NLS and sine-Gordon steps keep running as captured CUDA graphs while
 * profiling, with the events inside the graph; Navier-Stokes steps run as
 * direct launches while profiling.
 * pss_profile_read synchronises and writes 7 doubles:
 *   out[0] = kernel launches made by pss_step_n since profiling was switched on,
 *   out[1], out[2] = row passes timed and their total milliseconds,
 *   out[3], out[4] = column passes timed and their total milliseconds,
 *   out[5], out[6] = other step kernels (NS control) timed and total ms.
 * Switching profiling on clears the counters.  Errors: PSS_E_ARG (on < 0). */
int pss_set_profiling(pss_grid *g, int on);
int pss_profile_read(pss_grid *g, double *out, int cap, int *count);

/* Wait for all work enqueued on the grid's stream; reports deferred errors:
 * PSS_E_NOT_CONVERGED (NS), and PSS_E_CUDA when a column pass gave up waiting
 * for one of its tile copies (its bounded wait ran out): the state is then
 * lost and must be set again before the next step. */
int pss_sync(pss_grid *g);

/* Free every resource of the grid.  Safe on NULL. */
int pss_destroy(pss_grid *g);

/* Message of the last error on g (or of the last failed create when g is
 * NULL).  The string is owned by the library. */
const char *pss_last_error(const pss_grid *g);

/* In-place 2D complex FFT of `batch` device arrays [batch][ny][nx] (row FFTs,
 * then column FFTs), the building block of every step (Section 4).
 * direction -1: unnormalised forward transform, exponent sign -1;
 * direction +1: inverse including the factor 1/(nx ny).
 * data is a device pointer to interleaved complex of the given precision;
 * stream is a cudaStream_t or NULL (legacy default stream).  The first call
 * for a given (n, precision, device) uploads its twiddle table, which is kept
 * until process exit.  Asynchronous.  Errors: PSS_E_ARG, PSS_E_OOM, PSS_E_CUDA. */
int pss_fft2d(void *data, int64_t nx, int64_t ny, int64_t batch, int precision, int direction,
              void *stream);

/* Mass and energy of NLS fields (the diagnostics of pss_conserved_quantities
 * for PSS_EQ_NLS) from caller-owned device arrays, without allocating any
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc, such as code whose device memory belongs to
 * another allocator or a fixed budget, or latency-critical loops in which an
 * allocation, which may synchronise the device, is not acceptable.
 *  psi:     device, physical field, interleaved complex [batch][ny][nx];
 *  psi_hat: device, its unnormalised forward 2D DFT (e.g. pss_fft2d, -1);
 *  precision PSS_FP32 (complex64 inputs) or PSS_FP64 (complex128);
 *  out:     device, 2*batch doubles: out[2f] = mass, out[2f+1] = energy;
 *  stream:  cudaStream_t or NULL.  Asynchronous; read out after the stream.
 * Scratch lives in a static device array of the library sized for at most
 * 64 fields (198,144 bytes, held on every GPU that loads the library until
 * the process exits).  Every call shares that array: calls that overlap on
 * the GPU race on it, so serialise them (one stream, or events).  The first
 * call on each device looks up the array's device address with that device
 * current (again after the device's context changes, e.g. after
 * cudaDeviceReset); make that first call before any stream capture.
 * Errors: PSS_E_ARG (bad pointer, size, precision, or batch > 64, with a
 * message in pss_last_error(NULL)); PSS_E_CUDA if a CUDA error was already
 * pending on entry (nothing is launched) or a launch fails (the message
 * names which). */
int pss_nls_invariants_static(const void *psi, const void *psi_hat, int64_t nx, int64_t ny,
                              int64_t batch, double lx, double ly, double sigma, int precision,
                              double *out, void *stream);

/* Fused multiply-add rate of the current device in GFLOP/s (2 flops per FMA),
 * the peak that arithmetic-bound passes are compared with.  The paper has no
 * counterpart.  kind 0: FP32 FMA; 1: FP64 FMA; 2: FP32 FMA on packed pairs
 * (two FMAs per instruction).  One launch of independent FMA chains (8 CTAs
 * of 256 threads per SM), timed with CUDA events on `stream` (NULL: the
 * legacy default stream), best of three after a warm-up; synchronises the
 * stream.  Allocates nothing.  Errors: PSS_E_ARG, PSS_E_CUDA. */
int pss_fma_rate(int kind, double *gflops, void *stream);

/* Library version string. */
const char *pss_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSS_H */
