// Deterministic FP64 reductions for the conserved quantities.
//
// Every field is summed by RED_BLOCKS blocks of RED_THREADS threads with a
// fixed grid-stride assignment; each block folds its threads in a fixed tree
// and writes one partial, and a second kernel folds the partials in a fixed
// tree.  The result therefore does not depend on scheduling or on the batch.
#include <math.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fft_core.cuh"

namespace pss {

template <int K> __device__ __forceinline__ void block_sum(double (&a)[K], double *sh)
{
    // sh: K * RED_THREADS doubles
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * RED_THREADS + threadIdx.x] = a[k];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w)
#pragma unroll
            for (int k = 0; k < K; ++k)
                sh[k * RED_THREADS + threadIdx.x] += sh[k * RED_THREADS + threadIdx.x + w];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = sh[k * RED_THREADS];
}

// partials [batch][RED_BLOCKS][K] -> out [batch][K]
template <int K> __global__ void __launch_bounds__(RED_THREADS) k_fold(const double *partials, double *out)
{
    __shared__ double sh[K * RED_THREADS];
    const int64_t f = blockIdx.x;
    double a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS)
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] += partials[(f * RED_BLOCKS + i) * K + k];
    block_sum<K>(a, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) out[f * K + k] = a[k];
}

// NLS: sum |psi|^2, sum |psi|^4 (physical) and sum |k|^2 |psi_hat|^2 (spectral)
template <class Rl>
__global__ void __launch_bounds__(RED_THREADS)
    k_nls_sums(const V2<Rl> *psi, const V2<Rl> *hat, int64_t nx, int64_t ny,
               const double *kx2, const double *ky2, double *partials)
{
    __shared__ double sh[3 * RED_THREADS];
    const int64_t f = blockIdx.y, n = nx * ny;
    const int lgx = __ffsll(nx) - 1;  // nx is a power of two
    const V2<Rl> *p = psi + f * n, *h = hat + f * n;
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * RED_THREADS + threadIdx.x; i < n;
         i += int64_t(RED_BLOCKS) * RED_THREADS) {
        const V2<Rl> z = p[i];
        const double m2 = double(z.x) * z.x + double(z.y) * z.y;
        a[0] += m2;
        a[1] += m2 * m2;
        const V2<Rl> w = h[i];
        a[2] += (kx2[i & (nx - 1)] + ky2[i >> lgx]) * (double(w.x) * w.x + double(w.y) * w.y);
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) partials[(f * RED_BLOCKS + blockIdx.x) * 3 + k] = a[k];
}

template <class Rl>
cudaError_t nls_sums(const V2<Rl> *psi, const V2<Rl> *psi_hat, int64_t nx, int64_t ny,
                     int64_t batch, const double *kx2, const double *ky2, double *partials,
                     double *out, cudaStream_t s)
{
    k_nls_sums<Rl><<<dim3(RED_BLOCKS, unsigned(batch)), RED_THREADS, 0, s>>>(psi, psi_hat, nx, ny,
                                                                            kx2, ky2, partials);
    k_fold<3><<<unsigned(batch), RED_THREADS, 0, s>>>(partials, out);
    return cudaGetLastError();
}

// SG at t_{n-1/2}: X = u^n, Y = u^n - u^{n-1} (physical, real parts), U = uhat^n,
// D = uhat^n - uhat^{n-1}.  Sums: (Y/dt)^2 / 2, 1 - cos(ubar) = 2 sin^2(ubar/2)
// with ubar = X - Y/2, and |k|^2 |U - D/2|^2 (the spectrum of ubar).
template <class Rl>
__global__ void __launch_bounds__(RED_THREADS)
    k_sg_sums(const V2<Rl> *X, const V2<Rl> *Y, const V2<Rl> *U, const V2<Rl> *D, int64_t nx, int64_t ny,
              const double *kx2, const double *ky2, double dt, double *partials)
{
    __shared__ double sh[3 * RED_THREADS];
    const int64_t f = blockIdx.y, n = nx * ny, o = f * n;
    const int lgx = __ffsll(nx) - 1;  // nx is a power of two
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * RED_THREADS + threadIdx.x; i < n;
         i += int64_t(RED_BLOCKS) * RED_THREADS) {
        const double du = double(Y[o + i].x), ub = double(X[o + i].x) - 0.5 * du;
        const double sh2 = sin(0.5 * ub);
        a[0] += 0.5 * (du / dt) * (du / dt);
        a[1] += 2.0 * sh2 * sh2;
        const V2<Rl> u = U[o + i], d = D[o + i];
        const double br = double(u.x) - 0.5 * double(d.x), bi = double(u.y) - 0.5 * double(d.y);
        a[2] += (kx2[i & (nx - 1)] + ky2[i >> lgx]) * (br * br + bi * bi);
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) partials[(f * RED_BLOCKS + blockIdx.x) * 3 + k] = a[k];
}

// NS from the spectrum w_hat of each field (buffer fs[f].idx): Re w_hat(0,0)
// (= sum of w), sum |w_hat|^2, sum over k != 0 of |w_hat|^2 / |k|^2.
struct NsFieldRd {
    int idx, active, nonconv, pad;
    long long updates;
};
template <class Rl>
__global__ void __launch_bounds__(RED_THREADS)
    k_ns_sums(const NsFieldRd *fs, const V2<Rl> *w0, const V2<Rl> *w1, const V2<Rl> *w2, int64_t nx, int64_t ny,
              const double *kx2, const double *ky2, double *partials)
{
    __shared__ double sh[3 * RED_THREADS];
    const int64_t f = blockIdx.y, n = nx * ny;
    const int lgx = __ffsll(nx) - 1;  // nx is a power of two
    const int b = fs[f].idx;
    const V2<Rl> *w = (b == 0 ? w0 : b == 1 ? w1 : w2) + f * n;
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * RED_THREADS + threadIdx.x; i < n;
         i += int64_t(RED_BLOCKS) * RED_THREADS) {
        const V2<Rl> z = w[i];
        const double m2 = double(z.x) * z.x + double(z.y) * z.y;
        const double k2 = kx2[i & (nx - 1)] + ky2[i >> lgx];
        if (i == 0) a[0] += double(z.x);
        a[1] += m2;
        if (k2 > 0) a[2] += m2 / k2;
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) partials[(f * RED_BLOCKS + blockIdx.x) * 3 + k] = a[k];
}

template <class Rl>
cudaError_t sg_sums(const V2<Rl> *X, const V2<Rl> *Y, const V2<Rl> *U, const V2<Rl> *D, int64_t nx, int64_t ny,
                    int64_t batch, const double *kx2, const double *ky2, double dt, double *partials, double *out,
                    cudaStream_t s)
{
    k_sg_sums<Rl><<<dim3(RED_BLOCKS, unsigned(batch)), RED_THREADS, 0, s>>>(X, Y, U, D, nx, ny, kx2, ky2, dt,
                                                                           partials);
    k_fold<3><<<unsigned(batch), RED_THREADS, 0, s>>>(partials, out);
    return cudaGetLastError();
}

template <class Rl>
cudaError_t ns_sums(const void *fs, V2<Rl> *const w[3], int64_t nx, int64_t ny, int64_t batch, const double *kx2,
                    const double *ky2, double *partials, double *out, cudaStream_t s)
{
    k_ns_sums<Rl><<<dim3(RED_BLOCKS, unsigned(batch)), RED_THREADS, 0, s>>>(
        static_cast<const NsFieldRd *>(fs), w[0], w[1], w[2], nx, ny, kx2, ky2, partials);
    k_fold<3><<<unsigned(batch), RED_THREADS, 0, s>>>(partials, out);
    return cudaGetLastError();
}

template cudaError_t sg_sums<float>(const float2 *, const float2 *, const float2 *, const float2 *, int64_t,
                                    int64_t, int64_t, const double *, const double *, double, double *, double *,
                                    cudaStream_t);
template cudaError_t sg_sums<double>(const double2 *, const double2 *, const double2 *, const double2 *, int64_t,
                                     int64_t, int64_t, const double *, const double *, double, double *,
                                     double *, cudaStream_t);
template cudaError_t ns_sums<float>(const void *, float2 *const[3], int64_t, int64_t, int64_t, const double *,
                                    const double *, double *, double *, cudaStream_t);
template cudaError_t ns_sums<double>(const void *, double2 *const[3], int64_t, int64_t, int64_t, const double *,
                                     const double *, double *, double *, cudaStream_t);

template cudaError_t nls_sums<float>(const float2 *, const float2 *, int64_t, int64_t, int64_t,
                                     const double *, const double *, double *, double *,
                                     cudaStream_t);
template cudaError_t nls_sums<double>(const double2 *, const double2 *, int64_t, int64_t, int64_t,
                                      const double *, const double *, double *, double *,
                                      cudaStream_t);

}  // namespace pss

// ----------------------------------------------------------------------------
// NLS invariants without allocation.
//
// The same reduction as nls_sums (fixed block/thread assignment, fixed fold
// order), with |k|^2 formed from the index instead of a grid's table, and
// with the per-block partial sums and the per-field totals kept in one
// file-scope device array instead of memory a grid allocated.  It is for
// callers that cannot call cudaMalloc: code whose device memory is owned by
// another allocator or a fixed budget, and latency-critical loops where an
// allocation (which may synchronise the device) is not acceptable.  Every GPU
// that loads the library holds the array until the process exits, and every
// call shares it: calls that overlap on the GPU race on it.

namespace pss {

constexpr int STATIC_MAX_BATCH = 64;
constexpr size_t STATIC_PARTIALS = size_t(STATIC_MAX_BATCH) * RED_BLOCKS * 3;
constexpr size_t STATIC_DOUBLES = STATIC_PARTIALS + size_t(STATIC_MAX_BATCH) * 3;

// 64 fields * 128 blocks * 3 partial sums + 64 * 3 totals = 198,144 bytes
static __device__ __align__(256) double g_static_scratch[STATIC_DOUBLES];

namespace {
std::mutex g_static_mu;
// device address of g_static_scratch per device ordinal, with the context it
// was looked up in (a cudaDeviceReset gives the device a new primary context,
// in which the module and its array are loaded again)
struct StaticAddr {
    void *ctx = nullptr;
    double *ptr = nullptr;
};
StaticAddr g_static_addr[64];

// the driver's cuCtxGetCurrent, looked up once through the runtime (the
// library does not link the driver library itself)
using CtxGetCurrent = int (*)(void **);
CtxGetCurrent ctx_get_current()
{
    static const CtxGetCurrent fn = []() -> CtxGetCurrent {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<CtxGetCurrent>(p) : nullptr;
    }();
    return fn;
}

// Host code sees g_static_scratch only as a host-side stand-in; the device
// address is looked up once per device and context, with that device current.
cudaError_t static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const CtxGetCurrent get = ctx_get_current();
    if (!get) return cudaErrorNotSupported;
    void *ctx = nullptr;
    if (get(&ctx) != 0) return cudaErrorUnknown;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticAddr &a = g_static_addr[dev];
    if (!a.ptr || !ctx || a.ctx != ctx) {
        // the lookup also makes the device's primary context current if no
        // context was yet; the handle is read again after it
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        if (get(&ctx) != 0 || !ctx) return cudaErrorUnknown;
        a.ptr = static_cast<double *>(p);
        a.ctx = ctx;
    }
    *out = a.ptr;
    return cudaSuccess;
}

__device__ __forceinline__ double wavenumber2(int64_t m, int64_t n, double dk)
{
    const double k = dk * double(m < n / 2 ? m : m - n);
    return k * k;
}
}  // namespace

template <class Rl>
__global__ void __launch_bounds__(RED_THREADS)
    k_nls_sums_inline(const V2<Rl> *psi, const V2<Rl> *hat, int64_t nx, int64_t ny, double dkx,
                      double dky, double *partials)
{
    __shared__ double sh[3 * RED_THREADS];
    const int64_t f = blockIdx.y, n = nx * ny;
    const int lgx = __ffsll(nx) - 1;  // nx is a power of two
    const V2<Rl> *p = psi + f * n, *h = hat + f * n;
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * RED_THREADS + threadIdx.x; i < n;
         i += int64_t(RED_BLOCKS) * RED_THREADS) {
        const V2<Rl> z = p[i];
        const double m2 = double(z.x) * z.x + double(z.y) * z.y;
        a[0] += m2;
        a[1] += m2 * m2;
        const V2<Rl> w = h[i];
        a[2] += (wavenumber2(i & (nx - 1), nx, dkx) + wavenumber2(i >> lgx, ny, dky)) *
                (double(w.x) * w.x + double(w.y) * w.y);
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) partials[(f * RED_BLOCKS + blockIdx.x) * 3 + k] = a[k];
}

__global__ void k_nls_finish(const double *sums, int64_t batch, double dA, double inv_n,
                             double sigma, double *out)
{
    const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= batch) return;
    const double *s = sums + 3 * f;
    out[2 * f] = dA * s[0];
    out[2 * f + 1] = dA * (0.5 * s[2] * inv_n + 0.25 * sigma * s[1]);
}

}  // namespace pss

extern "C" int pss_nls_invariants_static(const void *psi, const void *psi_hat, int64_t nx,
                                         int64_t ny, int64_t batch, double lx, double ly,
                                         double sigma, int precision, double *out, void *stream)
{
    using namespace pss;
    auto ok = [](int64_t n) { return n >= 16 && n <= 8192 && (n & (n - 1)) == 0; };
    if (!psi || !psi_hat || !out || !ok(nx) || !ok(ny) || !(lx > 0) || !(ly > 0) ||
        !std::isfinite(sigma) || (precision != 0 && precision != 1)) {
        set_global_error("pss_nls_invariants_static: invalid argument");
        return 1;  // PSS_E_ARG
    }
    if (batch < 1 || batch > STATIC_MAX_BATCH) {
        set_global_error("pss_nls_invariants_static: batch must be in [1, 64], the size of the "
                         "library's static scratch");
        return 1;  // PSS_E_ARG
    }
    // an error left pending by earlier, unrelated work on this thread would
    // otherwise be reported (and cleared) as this call's launch failure
    if (cudaPeekAtLastError() != cudaSuccess) {
        set_global_error("pss_nls_invariants_static: a CUDA error was already pending before the call");
        return 3;  // PSS_E_CUDA
    }
    double *scratch = nullptr;
    if (static_scratch(&scratch) != cudaSuccess) {
        set_global_error("pss_nls_invariants_static: cudaGetSymbolAddress failed");
        return 3;  // PSS_E_CUDA
    }
    // every partial and total read below is first written by this same call,
    // so nothing has to be cleared between calls
    double *partials = scratch, *sums = scratch + STATIC_PARTIALS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double two_pi = 6.283185307179586476925286766559;
    const dim3 grid(RED_BLOCKS, unsigned(batch));
    auto launched = [](const char *what) {
        if (cudaGetLastError() == cudaSuccess) return true;
        char msg[128];
        snprintf(msg, sizeof msg, "pss_nls_invariants_static: launch of %s failed", what);
        set_global_error(msg);
        return false;
    };
    if (precision == 0)
        k_nls_sums_inline<float><<<grid, RED_THREADS, 0, s>>>(
            static_cast<const float2 *>(psi), static_cast<const float2 *>(psi_hat), nx, ny,
            two_pi / lx, two_pi / ly, partials);
    else
        k_nls_sums_inline<double><<<grid, RED_THREADS, 0, s>>>(
            static_cast<const double2 *>(psi), static_cast<const double2 *>(psi_hat), nx, ny,
            two_pi / lx, two_pi / ly, partials);
    if (!launched("the block sums")) return 3;  // PSS_E_CUDA
    k_fold<3><<<unsigned(batch), RED_THREADS, 0, s>>>(partials, sums);
    if (!launched("the fold")) return 3;
    k_nls_finish<<<1, 64, 0, s>>>(sums, batch, (lx / double(nx)) * (ly / double(ny)),
                                  1.0 / (double(nx) * double(ny)), sigma, out);
    if (!launched("the final scaling")) return 3;
    return 0;
}
