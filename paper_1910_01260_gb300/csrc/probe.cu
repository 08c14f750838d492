// FP64 fused multiply-add throughput of the current device: the measured
// peak against which the library's FP64-bound kernels (the full-order
// march, the reduced LU, the middle-matrix SVD) are reported.
#include "internal.h"

namespace {

constexpr int kChains = 16;  // independent FMA chains per thread (covers the pipe latency)

__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, double x, double y, double* sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 4
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    // the chains converge to y / (1 - x); writing the sum keeps them alive
    if (s == 12345.678) sink[0] = s;
}

}  // namespace

extern "C" st_status st_probe_fp64_fma(int32_t blocks_per_sm, int64_t iters, double* tflops, double* ms) {
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || !tflops)
        return st_fail(ST_ERR_ARG, "st_probe_fp64_fma: bad arguments");
    int dev = 0, sms = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    ST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ST_CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(sink);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return st_fail(ST_ERR_CUDA, "st_probe_fp64_fma: event creation failed");
    }
    const int blocks = blocks_per_sm * sms, threads = 256;
    // x < 1 keeps the chains bounded; one untimed launch warms the clocks
    fma_probe_kernel<<<blocks, threads>>>(iters / 4 + 1, 0.9999999, 1e-7, sink);
    cudaEventRecord(e0);
    fma_probe_kernel<<<blocks, threads>>>(iters, 0.9999999, 1e-7, sink);
    cudaEventRecord(e1);
    st_count_launch();
    st_count_launch();
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cleanup();
    if (err != cudaSuccess) return st_fail(ST_ERR_CUDA, "st_probe_fp64_fma: %s", cudaGetErrorString(err));
    const double flops = 2.0 * kChains * (double)iters * threads * blocks;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return ST_OK;
}
