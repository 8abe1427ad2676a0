// Elementwise helpers for state set-up and read-back (off the stepping path).
#include <math.h>

#include "fft_core.cuh"

namespace pss {

// dst[i] = (f(src[i]), 0) with f = identity or sin
template <class Rl>
__global__ void k_real_to_complex(const Rl *src, V2<Rl> *dst, int64_t n, int apply_sin)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const Rl x = src[i];
        dst[i] = V2<Rl>{apply_sin ? Rl(sin(double(x))) : x, Rl(0)};
    }
}

// dst[i] = Re(a[i]) - c * Re(b[i])   (b may be null)
template <class Rl>
__global__ void k_complex_to_real(const V2<Rl> *a, const V2<Rl> *b, Rl c, Rl *dst, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = b ? a[i].x - c * b[i].x : a[i].x;
}

// Sine-Gordon start-up: with uhat^0 = F u0 in u, F v0 in d and F sin u0 in s,
//   d^0 = uhat^0 - uhat^{-1} = dt F v0 + (dt^2/2) (|k|^2 uhat^0 + F sin u0)
// (backward Taylor step u^{-1} = u^0 - dt v0 + dt^2/2 (Lap u^0 - sin u^0)).
template <class Rl>
__global__ void k_sg_init(const V2<Rl> *u, V2<Rl> *d, const V2<Rl> *s, const double *kx2, const double *ky2,
                          double dt, int64_t nx, int64_t ny, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = i % nx, y = (i / nx) % ny;
        const double k2 = kx2[x] + ky2[y];
        const double h = 0.5 * dt * dt;
        d[i] = V2<Rl>{Rl(dt * double(d[i].x) + h * (k2 * double(u[i].x) + double(s[i].x))),
                      Rl(dt * double(d[i].y) + h * (k2 * double(u[i].y) + double(s[i].y)))};
    }
}

// copy every field's current vorticity (buffer fs[f].idx) into dst
struct NsFieldView {
    int idx, active, nonconv, pad;
    long long updates;
};
template <class Rl>
__global__ void k_ns_gather(const NsFieldView *fs, const V2<Rl> *w0, const V2<Rl> *w1, const V2<Rl> *w2,
                            V2<Rl> *dst, int64_t per_field, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int b = fs[i / per_field].idx;
        dst[i] = (b == 0 ? w0 : b == 1 ? w1 : w2)[i];
    }
}

// dst = a - c b (complex)
template <class Rl> __global__ void k_axpy(const V2<Rl> *a, const V2<Rl> *b, Rl c, V2<Rl> *dst, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = V2<Rl>{a[i].x - c * b[i].x, a[i].y - c * b[i].y};
}

// spectrum *= keepx[x] keepy[y] (the 2/3 rule mask, 0 or 1)
template <class Rl>
__global__ void k_mask(V2<Rl> *a, const Rl *keepx, const Rl *keepy, int64_t nx, int64_t ny, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const Rl m = keepx[i % nx] * keepy[(i / nx) % ny];
        a[i] = V2<Rl>{a[i].x * m, a[i].y * m};
    }
}

static unsigned blocks_for(int64_t n) { return unsigned(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096); }

template <class Rl> cudaError_t real_to_complex(const Rl *src, V2<Rl> *dst, int64_t n, bool apply_sin, cudaStream_t s)
{
    k_real_to_complex<Rl><<<blocks_for(n), 256, 0, s>>>(src, dst, n, apply_sin ? 1 : 0);
    return cudaGetLastError();
}
template <class Rl>
cudaError_t complex_to_real(const V2<Rl> *a, const V2<Rl> *b, Rl c, Rl *dst, int64_t n, cudaStream_t s)
{
    k_complex_to_real<Rl><<<blocks_for(n), 256, 0, s>>>(a, b, c, dst, n);
    return cudaGetLastError();
}
template <class Rl>
cudaError_t sg_init(const V2<Rl> *u, V2<Rl> *d, const V2<Rl> *sn, const double *kx2, const double *ky2, double dt,
                    int64_t nx, int64_t ny, int64_t batch, cudaStream_t s)
{
    const int64_t n = nx * ny * batch;
    k_sg_init<Rl><<<blocks_for(n), 256, 0, s>>>(u, d, sn, kx2, ky2, dt, nx, ny, n);
    return cudaGetLastError();
}
template <class Rl>
cudaError_t ns_gather(const void *fs, V2<Rl> *const w[3], V2<Rl> *dst, int64_t per_field, int64_t batch,
                      cudaStream_t s)
{
    const int64_t n = per_field * batch;
    k_ns_gather<Rl><<<blocks_for(n), 256, 0, s>>>(static_cast<const NsFieldView *>(fs), w[0], w[1], w[2], dst,
                                                 per_field, n);
    return cudaGetLastError();
}

template <class Rl> cudaError_t cplx_axpy(const V2<Rl> *a, const V2<Rl> *b, Rl c, V2<Rl> *dst, int64_t n, cudaStream_t s)
{
    k_axpy<Rl><<<blocks_for(n), 256, 0, s>>>(a, b, c, dst, n);
    return cudaGetLastError();
}
template <class Rl>
cudaError_t apply_mask(V2<Rl> *a, const Rl *keepx, const Rl *keepy, int64_t nx, int64_t ny, int64_t batch, cudaStream_t s)
{
    const int64_t n = nx * ny * batch;
    k_mask<Rl><<<blocks_for(n), 256, 0, s>>>(a, keepx, keepy, nx, ny, n);
    return cudaGetLastError();
}

#define PSS_INST(Rl)                                                                                      \
    template cudaError_t cplx_axpy<Rl>(const V2<Rl> *, const V2<Rl> *, Rl, V2<Rl> *, int64_t, cudaStream_t); \
    template cudaError_t apply_mask<Rl>(V2<Rl> *, const Rl *, const Rl *, int64_t, int64_t, int64_t, cudaStream_t); \
    template cudaError_t real_to_complex<Rl>(const Rl *, V2<Rl> *, int64_t, bool, cudaStream_t);          \
    template cudaError_t complex_to_real<Rl>(const V2<Rl> *, const V2<Rl> *, Rl, Rl *, int64_t, cudaStream_t); \
    template cudaError_t sg_init<Rl>(const V2<Rl> *, V2<Rl> *, const V2<Rl> *, const double *, const double *, \
                                     double, int64_t, int64_t, int64_t, cudaStream_t);                     \
    template cudaError_t ns_gather<Rl>(const void *, V2<Rl> *const[3], V2<Rl> *, int64_t, int64_t, cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
