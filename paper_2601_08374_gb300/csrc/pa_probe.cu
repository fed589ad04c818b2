// Measured FMA rate of the CUDA cores (pa_measure_fma_rate): the peak that
// the element kernels, bound by FP64 or FP32 arithmetic, are compared with,
// measured on the part instead of derived from unit counts and clocks.
//
// Every thread runs kChains independent multiply-add chains for `iters`
// steps, so the FMA pipe is never waiting on a dependency; the grid fills
// every SM several times over.  The chains stay bounded (a contraction
// towards a fixed point), and their sum is stored so the compiler keeps
// every FMA.
#include <vector>

#include "pa_internal.h"

namespace pa {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T *out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same FMA work on paired instructions (__ffma2_rn): kChains / 2
// chains of float2 per thread.
__global__ void __launch_bounds__(kProbeThreads) fma2_probe_kernel(float *out, int iters, float b, float c)
{
    float2 a[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        a[k] = make_float2(float(threadIdx.x + 2 * k) * 1e-3f, float(threadIdx.x + 2 * k + 1) * 1e-3f);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += a[k].x + a[k].y;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, bool PAIRED = false>
int measure(double *tflops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    // FP64 runs at a small fraction of the FP32 rate: fewer steps keep the
    // probe near a tenth of a second either way
    const int iters = sizeof(T) == 8 ? 256 : 8192;
    T *out = nullptr;
    PA_CUDA_TRY(cudaMalloc(&out, sizeof(T) * (size_t)blocks * kProbeThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PA_OK;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = set_error(PA_ECUDA, "pa_measure_fma_rate: event creation failed");
    } else {
        for (int rep = 0; rep < 6 && rc == PA_OK; ++rep) {
            cudaEventRecord(e0, s);
            if constexpr (PAIRED) fma2_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.999f, 1e-4f);
            else fma_probe_kernel<T><<<blocks, kProbeThreads, 0, s>>>(out, iters, T(0.999), T(1e-4));
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_error(e, "pa_measure_fma_rate");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    const double fma = (double)blocks * kProbeThreads * iters * 16.0 * kChains;
    *tflops = 2.0 * fma / (best * 1e-3) / 1e12;
    return PA_OK;
}

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" int pa_measure_fma_rate(int precision, double *tflops, void *stream)
{
    if (!tflops) return set_error(PA_EINVAL, "pa_measure_fma_rate: null output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == PA_FP64) return measure<double>(tflops, s);
    if (precision == PA_FP32) return measure<float>(tflops, s);
    if (precision == PA_FMA_FP32X2) return measure<float, true>(tflops, s);
    return set_error(PA_EINVAL, "pa_measure_fma_rate: bad precision");
}
