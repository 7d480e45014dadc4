// nb_probe.cu -- FMA throughput probes (measurement aid, include/nb_probe.h).
#include <cuda_runtime.h>

#include "../../include/nb_probe.h"

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma(T *sink, int64_t iters, T b, T c) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
nb_status run(int64_t iters, cudaStream_t st, double *fps, double *sec) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NB_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NB_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma<T>, kThreads, 0) != cudaSuccess)
        return NB_ECUDA;
    const int blocks = sms * (occ > 0 ? occ : 1);
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks * kThreads) != cudaSuccess) return NB_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 keeps the chains finite; c keeps them from decaying to 0
    k_fma<T><<<blocks, kThreads, 0, st>>>(sink, iters / 8 + 1, (T)0.999999, (T)1e-3);  // warm-up
    cudaEventRecord(e0, st);
    k_fma<T><<<blocks, kThreads, 0, st>>>(sink, iters, (T)0.999999, (T)1e-3);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return NB_ECUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    if (fps) *fps = flops / (ms * 1e-3);
    if (sec) *sec = ms * 1e-3;
    return NB_OK;
}
}  // namespace

extern "C" nb_status nb_probe_fma_peak(int32_t precision, int64_t iters, void *stream,
                                       double *flops_per_s, double *seconds) {
    if (iters < 1) return NB_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == NB_FP64) return run<double>(iters, st, flops_per_s, seconds);
    if (precision == NB_FP32) return run<float>(iters, st, flops_per_s, seconds);
    return NB_EINVAL;
}
