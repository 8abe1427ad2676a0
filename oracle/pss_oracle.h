/*
 * FP64 CPU oracle for the 2D periodic Fourier pseudospectral time steppers of
 * Cloutier, Muite and Rigge (arXiv:1206.3215).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * restatement of what the paper computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Conventions (all functions):
 *   - complex arrays are C99 `double complex`, row-major [ny][nx], x fastest;
 *   - the box is [x0, x0+lx) x [y0, y0+ly) with nx*ny points, x_j = x0 + j*lx/nx;
 *   - wavenumber k_m = (2*pi/L) * m, m in {0..n/2-1, -n/2..-1};
 *   - forward transform is the unnormalised DFT (exponent sign -1), the
 *     inverse carries 1/(nx*ny);
 *   - return value 0 = success, negative = bad argument.
 */
#ifndef PSS_ORACLE_H
#define PSS_ORACLE_H

#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Fourier transforms (Section 4: derivatives by multiplication in Fourier space) ---- */
int orc_fft1d(double complex *a, long n, int sign);                       /* in place, radix-2 */
int orc_dft1d(const double complex *in, double complex *out, long n, int sign); /* O(n^2) */
int orc_fft2d(double complex *a, long nx, long ny, int sign);             /* rows then columns */
int orc_wavenumbers(long n, double L, double *k);                         /* k[m], length n */

/* ---- Cubic NLS, Eq. 1, split-step Fourier of Section 4.1 ---- */
/* sigma: i psi_t + Lap psi = sigma |psi|^2 psi.  merged=0: literal Strang step
 * L(dt/2) N(dt) L(dt/2) repeated; merged=1: L(dt/2) [N L(dt)]^(n-1) N L(dt/2). */
int orc_nls_run(double complex *psi, long nx, long ny, double lx, double ly,
                double dt, double sigma, long nsteps, int merged);
/* Eq. 2: mass = integral |psi|^2, energy = integral |grad psi|^2/2 + sigma |psi|^4/4 */
int orc_nls_invariants(const double complex *psi, long nx, long ny, double lx, double ly,
                       double sigma, double *mass, double *energy);

/* ---- Sine-Gordon, Eq. 3, semi-implicit leapfrog of Section 4.2 ---- */
int orc_sg_init(const double *u0, const double *v0, long nx, long ny, double lx, double ly,
                double dt, double complex *uhat_n, double complex *uhat_nm1);
int orc_sg_run(double complex *uhat_n, double complex *uhat_nm1, long nx, long ny,
               double lx, double ly, double dt, long nsteps);
int orc_sg_fields(const double complex *uhat_n, const double complex *uhat_nm1, long nx, long ny,
                  double *u_n, double *u_nm1);
int orc_sg_hamiltonian(const double complex *uhat_n, const double complex *uhat_nm1, long nx,
                       long ny, double lx, double ly, double dt, double *H);

/* ---- 2D Navier-Stokes, vorticity/streamfunction form, Crank-Nicolson with
 *      fixed-point iteration of Section 4.3 ---- */
int orc_ns_init(const double *w0, long nx, long ny, int dealias, double complex *what);
int orc_ns_jacobian(const double complex *what, long nx, long ny, double lx, double ly,
                    double *J);
/* Returns 0, or 1 if some step hit max_iter (the state is then the last iterate).
 * iters[s] (if non-NULL, length nsteps) receives the number of CN updates of step s. */
int orc_ns_run(double complex *what, long nx, long ny, double lx, double ly, double nu,
               double dt, double tol, long max_iter, int dealias, long nsteps, long *iters);
/* scheme 0 as above; scheme 1: implicit midpoint (Jacobian of (w^k + w^n)/2) */
int orc_ns_run_scheme(double complex *what, long nx, long ny, double lx, double ly, double nu,
                      double dt, double tol, long max_iter, int dealias, long nsteps, long *iters,
                      int scheme);
int orc_ns_field(const double complex *what, long nx, long ny, double *w);
/* circulation = integral w, enstrophy = integral w^2 / 2, energy = integral |u|^2 / 2 */
int orc_ns_invariants(const double complex *what, long nx, long ny, double lx, double ly,
                      double *circulation, double *enstrophy, double *energy);

/* threads used by the OpenMP loops (1 when built without OpenMP) */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
