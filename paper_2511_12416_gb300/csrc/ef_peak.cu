// Throughput microbenchmarks for the roofline denominators: FP32 FMA (scalar
// and packed FFMA2), FP64 FMA, and Philox4x32-10 blocks. Every thread runs
// independent dependency chains long enough to hide the pipe latency; the
// results feed a reduction so that none of the work is dead code. The paper
// has no counterpart: these measure the GB300 the kernels run on.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ef_common.cuh"
#include "ef_internal.h"
#include "extraferm.h"

namespace ef {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32(float* out, int iters, float a, float b) {
    float x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32x2(float* out, int iters, float a, float b) {
    float2 x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
                x[c] = __ffma2_rn(x[c], a2, b2);
#else
                x[c] = make_float2(fmaf(x[c].x, a2.x, b2.x), fmaf(x[c].y, a2.y, b2.y));
#endif
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c].x + x[c].y;
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f64(double* out, int iters, double a, double b) {
    double x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Philox4x32-10 blocks with all lanes busy: four independent counters per
// thread, the key fixed, the outputs folded into a running word.
__global__ void __launch_bounds__(kPeakThreads) k_peak_philox(uint32_t* out, int iters, uint32_t k0, uint32_t k1) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)c, tid, 7u), k0, k1);
            acc ^= u.x ^ u.y ^ u.z ^ u.w;
        }
    }
    if (acc == 0x12345678u) out[tid] = acc;
}

}  // namespace ef

namespace {
thread_local std::string g_peak_err;
}

// Measured rate (operations per second) of kind 0: FP32 FMA flops (scalar
// FFMA), 1: FP32 FMA flops (packed FFMA2), 2: FP64 FMA flops, 3: Philox4x32-10
// blocks; best of `reps` timed launches after one warm-up, on the current
// device, synchronous.
extern "C" int ef_measure_peak(int32_t kind, int32_t reps, double* rate) {
    if (!rate || kind < 0 || kind > 3) return EF_EINVAL;
    if (reps < 1) reps = 1;
    const int sms = ef::sm_count();
    const int blocks = sms * 8;
    const int nthreads = blocks * ef::kPeakThreads;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)nthreads * 8) != cudaSuccess) return EF_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = kind == 2 ? 2048 : kind == 3 ? 256 : 4096;
    double per_thread = 0.0;
    switch (kind) {
        case 0: per_thread = 2.0 * iters * 8 * ef::kPeakChains; break;
        case 1: per_thread = 4.0 * iters * 8 * ef::kPeakChains; break;
        case 2: per_thread = 2.0 * iters * ef::kPeakChains; break;
        default: per_thread = 4.0 * iters; break;
    }
    float best = 1e30f;
    int rc = EF_OK;
    for (int r = 0; r <= reps; ++r) {
        cudaEventRecord(e0);
        switch (kind) {
            case 0: ef::k_peak_f32<<<blocks, ef::kPeakThreads>>>((float*)buf, iters, 0.9999f, 1e-4f); break;
            case 1: ef::k_peak_f32x2<<<blocks, ef::kPeakThreads>>>((float*)buf, iters, 0.9999f, 1e-4f); break;
            case 2: ef::k_peak_f64<<<blocks, ef::kPeakThreads>>>((double*)buf, iters, 0.9999, 1e-4); break;
            default: ef::k_peak_philox<<<blocks, ef::kPeakThreads>>>((uint32_t*)buf, iters, 0x1234u, 0x5678u); break;
        }
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = EF_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return rc;
    *rate = per_thread * nthreads / (best * 1e-3);
    return EF_OK;
}
