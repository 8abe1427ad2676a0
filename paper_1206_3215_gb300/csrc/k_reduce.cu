// Deterministic FP64 reductions for the conserved quantities.
//
// Every field is summed by RED_BLOCKS blocks of RED_THREADS threads with a
// fixed grid-stride assignment; each block folds its threads in a fixed tree
// and writes one partial, and a second kernel folds the partials in a fixed
// tree.  The result therefore does not depend on scheduling or on the batch.
#include <math.h>

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
    const V2<Rl> *p = psi + f * n, *h = hat + f * n;
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * RED_THREADS + threadIdx.x; i < n;
         i += int64_t(RED_BLOCKS) * RED_THREADS) {
        const V2<Rl> z = p[i];
        const double m2 = double(z.x) * z.x + double(z.y) * z.y;
        a[0] += m2;
        a[1] += m2 * m2;
        const V2<Rl> w = h[i];
        a[2] += (kx2[i % nx] + ky2[i / nx]) * (double(w.x) * w.x + double(w.y) * w.y);
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

template cudaError_t nls_sums<float>(const float2 *, const float2 *, int64_t, int64_t, int64_t,
                                     const double *, const double *, double *, double *,
                                     cudaStream_t);
template cudaError_t nls_sums<double>(const double2 *, const double2 *, int64_t, int64_t, int64_t,
                                      const double *, const double *, double *, double *,
                                      cudaStream_t);

}  // namespace pss
