// Measured FMA throughput of the CUDA cores: the denominator of the
// determinant kernels' roofline (the Keldysh sums are bound by the FP64 or
// FP32 FMA pipes, not by memory or tensor cores).
//
// Every thread runs kChains independent multiply-add chains held in registers,
// a <- a * b + c with |b| < 1, so that nothing but FMAs is timed: no memory
// traffic, no dependent-latency stalls once enough warps are resident.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qqmc_internal.h"

using namespace qqmc;

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

template <class R>
__global__ void fma_peak_kernel(R *out, long long iters, R b, R c) {
    R a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma_r(a[k], b, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (R)-1) out[0] = s;  // keeps the chains live; never true for these operands
}

template <class R>
int run(double seconds, double *tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_fma_peak: device query");
    R *out = nullptr;
    e = cudaMalloc(&out, sizeof(R));
    if (e != cudaSuccess) return cuda_error(e, "qqmc_fma_peak: allocation");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const int threads = 256;
    const int blocks = sms * 8;  // 64 warps per SM
    const R b = (R)0.999999, c = (R)1e-6;
    long long iters = 64;
    double ms = 0.0;
    // grow the loop until one launch lasts a good fraction of the requested time
    for (int tries = 0; tries < 24; ++tries) {
        fma_peak_kernel<R><<<blocks, threads>>>(out, iters, b, c);
        e = cudaEventRecord(t0);
        fma_peak_kernel<R><<<blocks, threads>>>(out, iters, b, c);
        if (e == cudaSuccess) e = cudaEventRecord(t1);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) break;
        float f = 0.f;
        cudaEventElapsedTime(&f, t0, t1);
        ms = f;
        if (ms >= 250.0 * seconds || iters > (1ll << 40)) break;
        iters *= 2;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_fma_peak: launch");
    const double fmas = (double)blocks * threads * kChains * kUnroll * (double)iters;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return QQMC_OK;
}

}  // namespace

extern "C" int qqmc_fma_peak(int precision, double seconds, double *tflops) {
    if (!tflops || !(seconds > 0.0) || seconds > 60.0)
        return set_error(QQMC_E_INVAL, "qqmc_fma_peak: tflops must not be NULL and seconds in (0, 60]");
    if (precision == QQMC_PREC_FP64) return run<double>(seconds, tflops);
    if (precision == QQMC_PREC_MIXED) return run<float>(seconds, tflops);
    return set_error(QQMC_E_INVAL, "qqmc_fma_peak: precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
}
