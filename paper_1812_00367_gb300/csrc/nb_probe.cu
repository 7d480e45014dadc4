// nb_probe.cu -- FMA throughput probes (measurement aid, include/nb_probe.h).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/nb_probe.h"
#include "nb_internal.cuh"

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;

// Multiplies and adds that the compiler may not contract into FMAs.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// The same products and sums issued as fused multiply-adds (x*b - 0, x*1 + c)
// with the constants passed at run time, so no compiler can fold them back.
__device__ __forceinline__ double fma_ptx(double a, double b, double c) {
    double r;
    asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
    return r;
}

// Instruction streams per chain and iteration (8 independent chains/thread):
//   kPure: 1 FMA
//   kMix: 16 FMA + 6 multiplies + 5 adds (the FP64 evaluation's fused :
//         non-fused ratio), 27 instructions
//   kMixFma: kMix with the multiplies and adds issued as FMAs
//   kAdd / kMul: 1 add / 1 multiply
enum ProbeMode { kPure = 0, kMix = 1, kMixFma = 2, kAdd = 3, kMul = 4 };

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_fma(T *sink, int64_t iters, T b, T c, T one, T nzero) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int64_t it = 0; it < iters; ++it) {
        if constexpr (MODE == kPure) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
        } else if constexpr (MODE == kAdd) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = add_rn(acc[k], c);
        } else if constexpr (MODE == kMul) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = mul_rn(acc[k], b);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
                if (r < 6) {
#pragma unroll
                    for (int k = 0; k < kChains; ++k)
                        acc[k] = MODE == kMix ? mul_rn(acc[k], b) : fma_ptx(acc[k], b, nzero);
                }
                if (r < 5) {
#pragma unroll
                    for (int k = 0; k < kChains; ++k)
                        acc[k] = MODE == kMix ? add_rn(acc[k], c) : fma_ptx(acc[k], one, c);
                }
            }
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed two-lane FP32 FMA (fma.rn.f32x2, sm_100 and later): each chain is a
// pair of floats in one 64-bit register, one instruction per chain and step.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__global__ void __launch_bounds__(kThreads) k_fma2(float *sink, int64_t iters, float b, float c) {
    unsigned long long acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = pack2((float)(threadIdx.x + k), (float)k);
    const unsigned long long bb = pack2(b, b), cc = pack2(c, c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[k]));
        s += lo + hi;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

nb_status run_fma2(int64_t iters, cudaStream_t st, double *fps, double *sec) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NB_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NB_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma2, kThreads, 0) != cudaSuccess)
        return NB_ECUDA;
    const int blocks = sms * (occ > 0 ? occ : 1);
    float *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * blocks * kThreads) != cudaSuccess) return NB_ECUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma2<<<blocks, kThreads, 0, st>>>(sink, iters / 8 + 1, 0.999999f, 1e-3f);  // warm-up
        e = cudaEventRecord(e0, st);
    }
    if (e == cudaSuccess) {
        k_fma2<<<blocks, kThreads, 0, st>>>(sink, iters, 0.999999f, 1e-3f);
        e = cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return NB_ECUDA;
    // two lanes x 2 flops per instruction
    const double flops = 4.0 * kChains * (double)iters * (double)blocks * kThreads;
    if (fps) *fps = flops / (ms * 1e-3);
    if (sec) *sec = ms * 1e-3;
    return NB_OK;
}

template <typename T, int MODE>
nb_status run(int64_t iters, cudaStream_t st, double *fps, double *sec) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NB_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NB_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma<T, MODE>, kThreads, 0) != cudaSuccess)
        return NB_ECUDA;
    const int blocks = sms * (occ > 0 ? occ : 1);
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks * kThreads) != cudaSuccess) return NB_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 keeps the chains finite; c keeps them from decaying to 0
    const T b = (T)0.999999, c = (T)1e-3, one = (T)1, nzero = -(T)0;
    k_fma<T, MODE><<<blocks, kThreads, 0, st>>>(sink, iters / 8 + 1, b, c, one, nzero);  // warm-up
    cudaEventRecord(e0, st);
    k_fma<T, MODE><<<blocks, kThreads, 0, st>>>(sink, iters, b, c, one, nzero);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return NB_ECUDA;
    // instructions x 2: an FMA-equivalent rate, comparable across modes
    const double per_iter = (MODE == kMix || MODE == kMixFma) ? 27.0 : 1.0;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads * per_iter;
    if (fps) *fps = flops / (ms * 1e-3);
    if (sec) *sec = ms * 1e-3;
    return NB_OK;
}
}  // namespace

extern "C" nb_status nb_probe_fma_peak(int32_t precision, int64_t iters, void *stream,
                                       double *flops_per_s, double *seconds) {
    if (iters < 1) return NB_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (precision) {
    case NB_FP64: return run<double, kPure>(iters, st, flops_per_s, seconds);
    case NB_FP32: return run<float, kPure>(iters, st, flops_per_s, seconds);
    case 3: return run<double, kMix>(iters, st, flops_per_s, seconds);
    case 4: return run<double, kMixFma>(iters, st, flops_per_s, seconds);
    case 5: return run<double, kAdd>(iters, st, flops_per_s, seconds);
    case 6: return run<double, kMul>(iters, st, flops_per_s, seconds);
    case 7: return run_fma2(iters, st, flops_per_s, seconds);
    default: break;
    }
    return NB_EINVAL;
}

// ------------------------------------------------------------------------
// Failure-detection self-test: the bounded mbarrier wait of the evaluation
// kernel, run against a barrier whose transaction count nothing will ever
// satisfy.  The wait gives up after its budget, records the timeout bit in a
// device word, and the kernel returns normally: no fault, no hang, the
// context stays usable.
#include "nb_internal.cuh"

namespace {
__global__ void k_selftest_wait(unsigned long long budget_ns, uint32_t *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        nb::mbar_init(&bar, 1);
        nb::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) nb::mbar_expect_tx(&bar, 16);  // 16 bytes that never arrive
    __syncthreads();
    const bool ok = nb::mbar_wait_bounded(&bar, 0, budget_ns);
    if (!ok && threadIdx.x == 0) atomicOr(err, nb::kErrTimeout);
}
}  // namespace

extern "C" nb_status nb_selftest_wait_timeout(double budget_seconds, void *stream) {
    if (!(budget_seconds > 0.0) || budget_seconds > 2.0) return NB_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(uint32_t)) != cudaSuccess) return NB_ENOMEM;
    uint32_t h_err = 0;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 64, 0, st>>>((unsigned long long)(budget_seconds * 1e9), d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_err);
    if (e != cudaSuccess) return NB_ECUDA;
    return (h_err & nb::kErrTimeout) ? NB_ETIMEOUT : NB_OK;
}

// ------------------------------------------------ reciprocal square roots
namespace {
__global__ void k_rsqrt(int which, const double *x, double *y, int64_t n, double neg_zero) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[k];
        if (which == 0) {
            y[k] = NB_FP64_RSQRT3 ? nb::rsqrt_f64_3(v, neg_zero) : nb::rsqrt_f64_fma(v, neg_zero);
        } else if (which == 2) {
            y[k] = nb::rsqrt_f64_fma(v, neg_zero);
        } else {
            nb::ff r2;
            r2.hi = __double2float_rn(v);
            r2.lo = __double2float_rn(v - (double)r2.hi);
            const nb::ff r = nb::rsqrt_ff(r2);
            y[k] = (double)r.hi + (double)r.lo;
        }
    }
}
}  // namespace

extern "C" nb_status nb_probe_rsqrt(int32_t which, const double *x, double *y, int64_t n,
                                    void *stream) {
    if (which < 0 || which > 2) return NB_EINVAL;
    if (n < 0 || (n > 0 && (!x || !y))) return NB_EINVAL;
    if (n == 0) return NB_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_rsqrt<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(which, x, y, n, -0.0);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ECUDA;
}
