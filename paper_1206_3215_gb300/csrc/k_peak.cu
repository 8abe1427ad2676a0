// Fused multiply-add rate of the device: the peak against which passes that
// are bound by arithmetic (the FP64 path) are measured.  Each thread runs
// CHAINS independent chains x <- x a + b, enough independent work per warp
// to keep the FMA pipe busy; the rate is the FMAs of one timed launch over
// its CUDA-event duration.
#include <cuda_runtime.h>

#include "../../include/pss.h"
#include "internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

// the chains' sum lands here (a device variable: nothing is allocated)
__device__ double g_fma_sink;

template <class T> __global__ void __launch_bounds__(THREADS) k_fma_chain(T a, T b, int iters)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == T(-1)) g_fma_sink = double(s);  // keeps the chains; the sum is never -1
}

// the same with packed pairs of FP32 values (two FMAs per instruction)
__global__ void __launch_bounds__(THREADS) k_fma2_chain(float2 a, float2 b, int iters)
{
    float2 x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = float2{float(threadIdx.x + c) * 1e-3f, float(c) * 1e-3f};
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = __ffma2_rn(x[c], a, b);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
    if (s == -1.0f) g_fma_sink = double(s);
}

}  // namespace

extern "C" int pss_fma_rate(int kind, double *gflops, void *stream)
{
    using namespace pss;
    if (!gflops || kind < 0 || kind > 2) {
        set_global_error("pss_fma_rate: invalid argument");
        return 1;  // PSS_E_ARG
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error("pss_fma_rate: no device");
        return 3;  // PSS_E_CUDA
    }
    // eight CTAs of 256 threads per SM (2048 threads, the SM's limit)
    const int blocks = 8 * sms;
    // about a millisecond or more per launch at the expected rates
    const int iters = kind == 1 ? 1024 : 16384;
    auto launch = [&]() {
        if (kind == 0)
            k_fma_chain<float><<<blocks, THREADS, 0, s>>>(0.999999f, 1e-6f, iters);
        else if (kind == 1)
            k_fma_chain<double><<<blocks, THREADS, 0, s>>>(0.999999999, 1e-9, iters);
        else
            k_fma2_chain<<<blocks, THREADS, 0, s>>>(float2{0.999999f, 0.999998f}, float2{1e-6f, 2e-6f}, iters);
        return cudaGetLastError();
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 0.0f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();  // warm-up
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        float ms = 0.0f;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess || (e = launch()) != cudaSuccess ||
            (e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (best == 0.0f || ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || !(best > 0.0f)) {
        set_global_error("pss_fma_rate: launch or timing failed");
        return 3;  // PSS_E_CUDA
    }
    const double fmas = double(blocks) * THREADS * CHAINS * double(iters) * (kind == 2 ? 2.0 : 1.0);
    *gflops = 2.0 * fmas / (double(best) * 1e-3) / 1e9;
    return 0;
}
