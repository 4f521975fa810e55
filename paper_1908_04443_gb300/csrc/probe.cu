// Rate probe of the FP64 pipe (no counterpart in the paper): the FP64 step kernels are bound by
// the FP64 arithmetic of GB300 rather than by HBM, and their roofline needs the device's measured
// FP64 FMA rate.  Every thread runs eight independent chains of fused multiply-adds
// a <- a * b + c (2 flops each) whose values stay bounded, on a grid of several waves.
#include <cuda_runtime.h>

#include "kernels.h"

namespace lbmwet {

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) dfma_chains(double* out, double b, double c, int iters) {
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1e-3 * (threadIdx.x + k);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 1234.5678) out[0] = s;   // keeps the chains live; never true for these values
}

}  // namespace

cudaError_t probe_fp64_rate(cudaStream_t s, double* gflops) {
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    double* d_out = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_out), sizeof(double), s);
    if (e != cudaSuccess) return e;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = sms * 16, threads = 256, iters = 4096;
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(t0, s);
        dfma_chains<<<blocks, threads, 0, s>>>(d_out, 0.999999999, 1e-9, iters);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        const double flops = 2.0 * CHAINS * double(iters) * blocks * threads;
        if (e == cudaSuccess && rep > 0 && ms > 0.0f) best = best > flops / (ms * 1e6) ? best : flops / (ms * 1e6);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFreeAsync(d_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *gflops = best;
    return e;
}

}  // namespace lbmwet
