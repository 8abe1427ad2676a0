/*
 * FP64 CPU oracle for arXiv:1206.3215 (Cloutier, Muite, Rigge): Fourier
 * pseudospectral time stepping of the 2D cubic NLS (Eq. 1, Section 4.1), the
 * sine-Gordon equation (Eq. 3, Section 4.2) and 2D Navier-Stokes in
 * vorticity/streamfunction form (Section 3.3, Section 4.3).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Every routine is the
 * plain definition or the paper's algorithm in the paper's order: a naive
 * iterative radix-2 FFT, explicit wavenumber loops, one pointwise loop per
 * formula.  No fusion, no blocking.  OpenMP only splits independent rows and
 * columns, so results do not depend on the thread count.  Reductions run
 * serially with Neumaier compensated summation.
 *
 * Readings where the paper is silent or inconsistent (each is also listed in
 * the design notes):
 *  - NLS sign: i psi_t + Lap psi = sigma |psi|^2 psi.  The nonlinear sub-step
 *    is psi <- exp(-i sigma |psi|^2 dt) psi and the energy carries
 *    +sigma |psi|^4 / 4 (Eq. 1 is sigma=+1; the printed sub-step and energy of
 *    Section 4.1 / Eq. 2 correspond to sigma=-1).
 *  - NLS half step: exp(-i |k|^2 dt/2) (Section 4.1 prints dt, the exact
 *    solution of the linear equation over dt/2 has dt/2).
 *  - SG: the average of the Laplacian enters with a minus sign so that the
 *    scheme discretises Eq. 3 (the printed "+" is ill posed).  Start-up by a
 *    second-order backward Taylor step; Hamiltonian at n-1/2 (see below).
 *  - NS: omega_t + psi_y omega_x - psi_x omega_y = nu Lap omega, Lap psi = -omega;
 *    trapezoidal Jacobian; the convergence test is the absolute
 *    integral of (omega^{k} - omega^{k+1})^2 (Parseval), the accepted state is
 *    the newest iterate; 2/3-rule square truncation 3|m| < n on J and on the
 *    initial vorticity when dealiasing is on; odd derivatives vanish at the
 *    Nyquist index when it is off.
 */
#include "pss_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation: a plain serial sum with an error term.  */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double ks_val(const ksum *k) { return k->s + k->c; }

/* ------------------------------------------------------------------------ */
/* 1D transforms                                                            */

/* Iterative radix-2 Cooley-Tukey, decimation in time: bit-reversal
 * permutation, then log2(n) levels of butterflies.  Twiddle for level `len`
 * and offset j is exp(sign * 2 pi i j / len) from libm cos/sin. */
int orc_fft1d(cplx *a, long n, int sign)
{
    if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
    for (long i = 1, j = 0; i < n; i++) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (long len = 2; len <= n; len <<= 1) {
        long half = len >> 1;
        for (long j = 0; j < half; j++) {
            double ang = sign * TWO_PI * (double)j / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (long s = 0; s < n; s += len) {
                cplx u = a[s + j];
                cplx v = a[s + j + half] * w;
                a[s + j] = u + v;
                a[s + j + half] = u - v;
            }
        }
    }
    return 0;
}

/* Brute-force DFT: out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
int orc_dft1d(const cplx *in, cplx *out, long n, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return -1;
    for (long k = 0; k < n; k++) {
        cplx acc = 0;
        for (long j = 0; j < n; j++) {
            long e = (j * k) % n; /* exact reduction of the angle */
            double ang = sign * TWO_PI * (double)e / (double)n;
            acc += in[j] * (cos(ang) + I * sin(ang));
        }
        out[k] = acc;
    }
    return 0;
}

/* 2D transform: 1D transform of every row (x), then of every column (y).
 * sign=-1 forward (unnormalised), sign=+1 inverse including 1/(nx ny). */
int orc_fft2d(cplx *a, long nx, long ny, int sign)
{
    if (!is_pow2(nx) || !is_pow2(ny) || (sign != 1 && sign != -1)) return -1;
    long y;
#pragma omp parallel for schedule(static)
    for (y = 0; y < ny; y++) orc_fft1d(a + y * nx, nx, sign);
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
        long x;
#pragma omp for schedule(static)
        for (x = 0; x < nx; x++) {
            for (long yy = 0; yy < ny; yy++) col[yy] = a[yy * nx + x];
            orc_fft1d(col, ny, sign);
            for (long yy = 0; yy < ny; yy++) a[yy * nx + x] = col[yy];
        }
        free(col);
    }
    if (sign == 1) {
        double s = 1.0 / ((double)nx * (double)ny);
        long i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < nx * ny; i++) a[i] *= s;
    }
    return 0;
}

int orc_wavenumbers(long n, double L, double *k)
{
    if (n < 1 || !(L > 0)) return -1;
    for (long m = 0; m < n; m++) {
        long ms = (m < n / 2) ? m : m - n; /* Nyquist m = n/2 maps to -n/2 */
        k[m] = TWO_PI / L * (double)ms;
    }
    return 0;
}

/* signed mode index of storage index m */
static long signed_mode(long m, long n) { return (m < n / 2) ? m : m - n; }

/* ------------------------------------------------------------------------ */
/* Cubic NLS (Eq. 1), Strang split-step Fourier (Section 4.1)              */

/* Linear sub-step in Fourier space: psi_hat <- exp(-i |k|^2 tau) psi_hat,
 * the exact solution of i psi_t + Lap psi = 0 over time tau. */
static void nls_linear(cplx *a, long nx, long ny, const double *kx, const double *ky, double tau)
{
    long y;
#pragma omp parallel for schedule(static)
    for (y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            a[y * nx + x] *= cexp(-I * k2 * tau);
        }
}

/* Nonlinear sub-step in physical space: i psi_t = sigma |psi|^2 psi has
 * |psi| constant, so psi(dt) = exp(-i sigma |psi|^2 dt) psi(0). */
static void nls_nonlinear(cplx *a, long n, double sigma, double dt)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; i++) {
        double m2 = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
        a[i] *= cexp(-I * sigma * m2 * dt);
    }
}

int orc_nls_run(cplx *psi, long nx, long ny, double lx, double ly, double dt, double sigma,
                long nsteps, int merged)
{
    if (!is_pow2(nx) || !is_pow2(ny) || nsteps < 0) return -1;
    if (nsteps == 0) return 0;
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    if (!merged) {
        for (long s = 0; s < nsteps; s++) {
            orc_fft2d(psi, nx, ny, -1);
            nls_linear(psi, nx, ny, kx, ky, 0.5 * dt);
            orc_fft2d(psi, nx, ny, +1);
            nls_nonlinear(psi, nx * ny, sigma, dt);
            orc_fft2d(psi, nx, ny, -1);
            nls_linear(psi, nx, ny, kx, ky, 0.5 * dt);
            orc_fft2d(psi, nx, ny, +1);
        }
    } else {
        /* consecutive half steps L(dt/2) L(dt/2) combine into L(dt) */
        orc_fft2d(psi, nx, ny, -1);
        nls_linear(psi, nx, ny, kx, ky, 0.5 * dt);
        for (long s = 0; s < nsteps; s++) {
            orc_fft2d(psi, nx, ny, +1);
            nls_nonlinear(psi, nx * ny, sigma, dt);
            orc_fft2d(psi, nx, ny, -1);
            nls_linear(psi, nx, ny, kx, ky, (s + 1 < nsteps) ? dt : 0.5 * dt);
        }
        orc_fft2d(psi, nx, ny, +1);
    }
    free(kx);
    free(ky);
    return 0;
}

/* Eq. 2.  Mass by the rectangle rule; the gradient term through Parseval
 * with the same |k|^2 as the propagator. */
int orc_nls_invariants(const cplx *psi, long nx, long ny, double lx, double ly, double sigma,
                       double *mass, double *energy)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    long n = nx * ny;
    double dA = (lx / nx) * (ly / ny);
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *hat = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    memcpy(hat, psi, sizeof(cplx) * (size_t)n);
    orc_fft2d(hat, nx, ny, -1);
    ksum m2 = {0, 0}, m4 = {0, 0}, g = {0, 0};
    for (long i = 0; i < n; i++) {
        double a2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        ks_add(&m2, a2);
        ks_add(&m4, a2 * a2);
    }
    for (long y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            cplx h = hat[y * nx + x];
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            ks_add(&g, k2 * (creal(h) * creal(h) + cimag(h) * cimag(h)));
        }
    *mass = dA * ks_val(&m2);
    *energy = dA * (0.5 * ks_val(&g) / (double)n + 0.25 * sigma * ks_val(&m4));
    free(hat);
    free(kx);
    free(ky);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sine-Gordon (Eq. 3), semi-implicit leapfrog (Section 4.2)                */
/* (u^{n+1} - 2u^n + u^{n-1})/dt^2 - Lap (u^{n+1} + 2u^n + u^{n-1})/4 = -sin u^n,
 * solved for u^{n+1} in Fourier space where Lap -> -|k|^2. */

static void real_to_hat(const double *u, cplx *hat, long nx, long ny)
{
    for (long i = 0; i < nx * ny; i++) hat[i] = u[i];
    orc_fft2d(hat, nx, ny, -1);
}

static void hat_to_real(const cplx *hat, double *u, cplx *work, long nx, long ny)
{
    memcpy(work, hat, sizeof(cplx) * (size_t)(nx * ny));
    orc_fft2d(work, nx, ny, +1);
    for (long i = 0; i < nx * ny; i++) u[i] = creal(work[i]);
}

int orc_sg_init(const double *u0, const double *v0, long nx, long ny, double lx, double ly,
                double dt, cplx *uhat_n, cplx *uhat_nm1)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    long n = nx * ny;
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *vhat = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *shat = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    real_to_hat(u0, uhat_n, nx, ny);
    real_to_hat(v0, vhat, nx, ny);
    for (long i = 0; i < n; i++) s[i] = sin(u0[i]);
    real_to_hat(s, shat, nx, ny);
    /* u^{-1} = u^0 - dt v^0 + dt^2/2 u_tt(0), with u_tt = Lap u - sin u */
    for (long y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            long i = y * nx + x;
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            uhat_nm1[i] = uhat_n[i] - dt * vhat[i] + 0.5 * dt * dt * (-k2 * uhat_n[i] - shat[i]);
        }
    free(vhat);
    free(shat);
    free(s);
    free(kx);
    free(ky);
    return 0;
}

int orc_sg_run(cplx *uhat_n, cplx *uhat_nm1, long nx, long ny, double lx, double ly, double dt,
               long nsteps)
{
    if (!is_pow2(nx) || !is_pow2(ny) || nsteps < 0) return -1;
    long n = nx * ny;
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (long s = 0; s < nsteps; s++) {
        /* u^n in physical space, then the explicit nonlinearity sin u^n */
        memcpy(work, uhat_n, sizeof(cplx) * (size_t)n);
        orc_fft2d(work, nx, ny, +1);
        long i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < n; i++) work[i] = sin(creal(work[i]));
        orc_fft2d(work, nx, ny, -1);
        long y;
#pragma omp parallel for schedule(static)
        for (y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long j = y * nx + x;
                double k2 = kx[x] * kx[x] + ky[y] * ky[y];
                cplx next = ((2.0 - 0.5 * dt * dt * k2) * uhat_n[j] - dt * dt * work[j]) /
                                (1.0 + 0.25 * dt * dt * k2) -
                            uhat_nm1[j];
                uhat_nm1[j] = uhat_n[j];
                uhat_n[j] = next;
            }
    }
    free(work);
    free(kx);
    free(ky);
    return 0;
}

int orc_sg_fields(const cplx *uhat_n, const cplx *uhat_nm1, long nx, long ny, double *u_n,
                  double *u_nm1)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)(nx * ny));
    hat_to_real(uhat_n, u_n, work, nx, ny);
    hat_to_real(uhat_nm1, u_nm1, work, nx, ny);
    free(work);
    return 0;
}

/* H at t_{n-1/2}: u_t by the difference (u^n - u^{n-1})/dt, the potential and
 * gradient at ubar = (u^n + u^{n-1})/2, the gradient term through Parseval.
 * For the linear part this is the quantity the scheme conserves exactly. */
int orc_sg_hamiltonian(const cplx *uhat_n, const cplx *uhat_nm1, long nx, long ny, double lx,
                       double ly, double dt, double *H)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    long n = nx * ny;
    double dA = (lx / nx) * (ly / ny);
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    double *un = (double *)malloc(sizeof(double) * (size_t)n);
    double *um = (double *)malloc(sizeof(double) * (size_t)n);
    cplx *bar = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    orc_sg_fields(uhat_n, uhat_nm1, nx, ny, un, um);
    ksum kin = {0, 0}, pot = {0, 0}, grad = {0, 0};
    for (long i = 0; i < n; i++) {
        double ut = (un[i] - um[i]) / dt;
        double ub = 0.5 * (un[i] + um[i]);
        ks_add(&kin, 0.5 * ut * ut);
        ks_add(&pot, 1.0 - cos(ub));
        bar[i] = ub;
    }
    orc_fft2d(bar, nx, ny, -1);
    for (long y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            cplx h = bar[y * nx + x];
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            ks_add(&grad, k2 * (creal(h) * creal(h) + cimag(h) * cimag(h)));
        }
    *H = dA * (ks_val(&kin) + ks_val(&pot)) + 0.5 * dA * ks_val(&grad) / (double)n;
    free(un);
    free(um);
    free(bar);
    free(kx);
    free(ky);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 2D Navier-Stokes (Section 3.3), Crank-Nicolson + fixed point (Section 4.3) */

/* 2/3 rule, square truncation: keep mode m iff 3|m| < n in both directions. */
static int keep_mode(long mx, long my, long nx, long ny)
{
    return 3 * labs(signed_mode(mx, nx)) < nx && 3 * labs(signed_mode(my, ny)) < ny;
}

int orc_ns_init(const double *w0, long nx, long ny, int dealias, cplx *what)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    real_to_hat(w0, what, nx, ny);
    if (dealias)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++)
                if (!keep_mode(x, y, nx, ny)) what[y * nx + x] = 0;
    return 0;
}

/* Wavenumber used for an odd (first) derivative: zero at the Nyquist index,
 * where the derivative of the interpolant of a real field is not real. */
static double odd_k(const double *k, long m, long n) { return (m == n / 2) ? 0.0 : k[m]; }

/* J = psi_y omega_x - psi_x omega_y in physical space, with Lap psi = -omega
 * (psi_hat = omega_hat / |k|^2, mean of psi zero); four inverse transforms,
 * one per derivative field. */
static void ns_jacobian_phys(const cplx *what, long nx, long ny, const double *kx,
                             const double *ky, double *J, cplx *d1, cplx *d2, cplx *d3, cplx *d4)
{
    for (long y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            long i = y * nx + x;
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            cplx ph = (k2 > 0) ? what[i] / k2 : 0;
            double ax = odd_k(kx, x, nx), ay = odd_k(ky, y, ny);
            d1[i] = I * ax * ph;      /* psi_x   */
            d2[i] = I * ay * ph;      /* psi_y   */
            d3[i] = I * ax * what[i]; /* omega_x */
            d4[i] = I * ay * what[i]; /* omega_y */
        }
    orc_fft2d(d1, nx, ny, +1);
    orc_fft2d(d2, nx, ny, +1);
    orc_fft2d(d3, nx, ny, +1);
    orc_fft2d(d4, nx, ny, +1);
    for (long i = 0; i < nx * ny; i++)
        J[i] = creal(d2[i]) * creal(d3[i]) - creal(d1[i]) * creal(d4[i]);
}

int orc_ns_jacobian(const cplx *what, long nx, long ny, double lx, double ly, double *J)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    long n = nx * ny;
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *d = (cplx *)malloc(sizeof(cplx) * (size_t)(4 * n));
    ns_jacobian_phys(what, nx, ny, kx, ky, J, d, d + n, d + 2 * n, d + 3 * n);
    free(d);
    free(kx);
    free(ky);
    return 0;
}

/* J_hat = D . F[J(omega_hat)] */
static void ns_jacobian_hat(const cplx *what, long nx, long ny, const double *kx,
                            const double *ky, int dealias, cplx *jhat, double *J, cplx *d)
{
    long n = nx * ny;
    ns_jacobian_phys(what, nx, ny, kx, ky, J, d, d + n, d + 2 * n, d + 3 * n);
    real_to_hat(J, jhat, nx, ny);
    if (dealias)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++)
                if (!keep_mode(x, y, nx, ny)) jhat[y * nx + x] = 0;
}

int orc_ns_run(cplx *what, long nx, long ny, double lx, double ly, double nu, double dt,
               double tol, long max_iter, int dealias, long nsteps, long *iters)
{
    return orc_ns_run_scheme(what, nx, ny, lx, ly, nu, dt, tol, max_iter, dealias, nsteps, iters, 0);
}

/* scheme 0: the paper's Crank-Nicolson diffusion with the trapezoidal
 * Jacobian (J^k + J^n)/2; scheme 1: implicit midpoint, the Jacobian of the
 * midpoint (w^k + w^n)/2 with the same Crank-Nicolson diffusion:
 *   (w^{k+1} - w^n)/dt - nu Lap (w^{k+1} + w^n)/2 + J((w^k + w^n)/2) = 0. */
int orc_ns_run_scheme(cplx *what, long nx, long ny, double lx, double ly, double nu, double dt,
                      double tol, long max_iter, int dealias, long nsteps, long *iters, int scheme)
{
    if (!is_pow2(nx) || !is_pow2(ny) || nsteps < 0 || max_iter < 1) return -1;
    long n = nx * ny;
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *jn = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *jk = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *wk = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *wk1 = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    double *J = (double *)malloc(sizeof(double) * (size_t)n);
    cplx *d = (cplx *)malloc(sizeof(cplx) * (size_t)(4 * n));
    /* integral of f^2 = (lx ly / n^2) sum |f_hat|^2 (Parseval) */
    double parseval = lx * ly / ((double)n * (double)n);
    int status = 0;
    for (long s = 0; s < nsteps; s++) {
        ns_jacobian_hat(what, nx, ny, kx, ky, dealias, jn, J, d);
        memcpy(wk, what, sizeof(cplx) * (size_t)n);
        long k = 0;
        int converged = 0;
        while (k < max_iter) {
            const cplx *jcur = jn;
            if (k > 0) {
                if (scheme == 1) {
                    /* the midpoint (w^k + w^n)/2 */
                    for (long i = 0; i < n; i++) wk1[i] = 0.5 * (wk[i] + what[i]);
                    ns_jacobian_hat(wk1, nx, ny, kx, ky, dealias, jk, J, d);
                } else {
                    ns_jacobian_hat(wk, nx, ny, kx, ky, dealias, jk, J, d);
                }
                jcur = jk;
            }
            ksum diff = {0, 0};
            for (long y = 0; y < ny; y++)
                for (long x = 0; x < nx; x++) {
                    long i = y * nx + x;
                    double a = 0.5 * dt * nu * (kx[x] * kx[x] + ky[y] * ky[y]);
                    if (scheme == 1) /* ... + J((w^k + w^n)/2) = 0 */
                        wk1[i] = ((1.0 - a) * what[i] - dt * jcur[i]) / (1.0 + a);
                    else /* ... + (J^k + J^n)/2 = 0 */
                        wk1[i] = ((1.0 - a) * what[i] - 0.5 * dt * (jcur[i] + jn[i])) / (1.0 + a);
                    cplx e = wk1[i] - wk[i];
                    ks_add(&diff, creal(e) * creal(e) + cimag(e) * cimag(e));
                }
            k++;
            memcpy(wk, wk1, sizeof(cplx) * (size_t)n);
            if (parseval * ks_val(&diff) < tol) {
                converged = 1;
                break;
            }
        }
        memcpy(what, wk, sizeof(cplx) * (size_t)n);
        if (iters) iters[s] = k;
        if (!converged) status = 1;
    }
    free(jn);
    free(jk);
    free(wk);
    free(wk1);
    free(J);
    free(d);
    free(kx);
    free(ky);
    return status;
}

int orc_ns_field(const cplx *what, long nx, long ny, double *w)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)(nx * ny));
    hat_to_real(what, w, work, nx, ny);
    free(work);
    return 0;
}

/* Rectangle-rule integrals of omega, omega^2/2 and (u^2+v^2)/2 with the
 * velocity (u, v) = (psi_y, -psi_x) formed in physical space. */
int orc_ns_invariants(const cplx *what, long nx, long ny, double lx, double ly,
                      double *circulation, double *enstrophy, double *energy)
{
    if (!is_pow2(nx) || !is_pow2(ny)) return -1;
    long n = nx * ny;
    double dA = (lx / nx) * (ly / ny);
    double *kx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ky = (double *)malloc(sizeof(double) * (size_t)ny);
    orc_wavenumbers(nx, lx, kx);
    orc_wavenumbers(ny, ly, ky);
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *u = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *v = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (long y = 0; y < ny; y++)
        for (long x = 0; x < nx; x++) {
            long i = y * nx + x;
            double k2 = kx[x] * kx[x] + ky[y] * ky[y];
            cplx ph = (k2 > 0) ? what[i] / k2 : 0;
            w[i] = what[i];
            u[i] = I * odd_k(ky, y, ny) * ph;  /* psi_y  */
            v[i] = -I * odd_k(kx, x, nx) * ph; /* -psi_x */
        }
    orc_fft2d(w, nx, ny, +1);
    orc_fft2d(u, nx, ny, +1);
    orc_fft2d(v, nx, ny, +1);
    ksum c = {0, 0}, z = {0, 0}, e = {0, 0};
    for (long i = 0; i < n; i++) {
        double wr = creal(w[i]), ur = creal(u[i]), vr = creal(v[i]);
        ks_add(&c, wr);
        ks_add(&z, 0.5 * wr * wr);
        ks_add(&e, 0.5 * (ur * ur + vr * vr));
    }
    *circulation = dA * ks_val(&c);
    *enstrophy = dA * ks_val(&z);
    *energy = dA * ks_val(&e);
    free(w);
    free(u);
    free(v);
    free(kx);
    free(ky);
    return 0;
}
