// gf_peak.cu -- gf_fma_peak: the measured arithmetic peak that the
// ALU-bound sweeps are reported against.  On this GPU the FP64 sweeps are
// bound by the small FP64 unit, not by HBM; their roofline needs the rate at
// which this GPU actually retires fused multiply-adds, measured the same way
// the sweeps are timed (CUDA events around kernel launches).
//
// The kernel runs, in every thread, eight independent chains of fused
// multiply-adds x <- x a + b (no data reuse, no memory traffic, enough
// warps per SM to hide the FMA latency), so its time is set by the FMA pipe
// alone.  One FMA counts as two floating-point operations.
#include <cuda_runtime.h>

#include "gf.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)c;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // never true for these inputs; keeps every chain alive without a store per thread
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int iters, double *tflops, double *ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return GF_ECUDA;
    const int blocks = 8 * sms;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GF_OK;
    float ms = 0.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GF_ECUDA;
    const T a = (T)0.999999, b = (T)1e-6;
    if (rc == GF_OK) {
        k_fma_chains<T><<<blocks, kThreads>>>(nullptr, iters, a, b);  // warm-up
        cudaEventRecord(e0);
        for (int r = 0; r < 3; ++r) k_fma_chains<T><<<blocks, kThreads>>>(nullptr, iters, a, b);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = GF_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != GF_OK || !(ms > 0.0f)) return GF_ECUDA;
    const double fmas = 3.0 * blocks * kThreads * (double)kChains * iters;
    if (tflops) *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms / 3.0;
    return GF_OK;
}

}  // namespace

extern "C" int gf_fma_peak(int fp64, int iters, double *tflops, double *ms_per_launch)
{
    if ((fp64 != 0 && fp64 != 1) || iters < 1) return GF_EINVAL;
    return fp64 ? measure<double>(iters, tflops, ms_per_launch) : measure<float>(iters, tflops, ms_per_launch);
}
