// FP32 multiply-add peak of the current GPU, measured.
//
// The detector is bound by single-precision FMA throughput, so its roofline
// denominator is measured here rather than taken from unit counts: a grid of
// 4 CTAs x 256 threads per SM runs independent FMA chains out of registers
// (no memory traffic inside the loop) and the launch is timed with CUDA
// events on the caller's stream.  Two forms: scalar FMAs (one multiply-add
// per lane and instruction) and packed two-lane FMAs (__ffma2_rn, two per
// lane and instruction).  Both do the same arithmetic per thread; the higher
// rate is the pipe's peak, the ratio shows whether packing saves issue slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dog.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;
constexpr int kChains = 16;   // independent scalar chains per thread (8 packed pairs)

template <bool PAIR>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float a, float b, long long iters, float* sink) {
    const float seed = (float)(threadIdx.x + blockIdx.x) * 1e-6f;
    float total = 0.0f;
    if (PAIR) {
        float2 acc[kChains / 2];
#pragma unroll
        for (int u = 0; u < kChains / 2; ++u) acc[u] = make_float2(seed + u, seed - u);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (long long it = 0; it < iters; ++it) {
#pragma unroll
            for (int rep = 0; rep < 4; ++rep)
#pragma unroll
                for (int u = 0; u < kChains / 2; ++u) acc[u] = __ffma2_rn(acc[u], a2, b2);
        }
#pragma unroll
        for (int u = 0; u < kChains / 2; ++u) total += acc[u].x + acc[u].y;
    } else {
        float acc[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) acc[u] = seed + u;
        for (long long it = 0; it < iters; ++it) {
#pragma unroll
            for (int rep = 0; rep < 4; ++rep)
#pragma unroll
                for (int u = 0; u < kChains; ++u) acc[u] = __fmaf_rn(acc[u], a, b);
        }
#pragma unroll
        for (int u = 0; u < kChains; ++u) total += acc[u];
    }
    // keeps the chains live; the condition never holds for the values used
    if (total == -1.0f) sink[0] = total;
}

}  // namespace

extern "C" int dog_fma_peak(int32_t pair, int64_t iters, int32_t reps, double* h_tflops, double* h_ms,
                            void* stream) {
    if (!h_tflops || iters < 1 || reps < 1) return DOG_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DOG_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return DOG_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DOG_OK;
    std::vector<float> ms;
    const int grid = sms * kCtasPerSm;
    auto launch = [&](long long n) {
        if (pair) fma_peak_kernel<true><<<grid, kThreads, 0, s>>>(0.9999999f, 1e-7f, n, sink);
        else fma_peak_kernel<false><<<grid, kThreads, 0, s>>>(0.9999999f, 1e-7f, n, sink);
        return cudaGetLastError();
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DOG_ERR_CUDA;
    } else if (launch(iters / 8 + 1) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        rc = DOG_ERR_CUDA;   // warm-up (clock ramp)
    } else {
        for (int r = 0; r < reps && rc == DOG_OK; ++r) {
            float t = 0.0f;
            if (cudaEventRecord(e0, s) != cudaSuccess || launch(iters) != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                rc = DOG_ERR_CUDA;
            else
                ms.push_back(t);
        }
    }
    if (rc == DOG_OK) {
        std::sort(ms.begin(), ms.end());
        const double med = ms[ms.size() / 2];
        // 4 repeats x 16 chains x 2 flop per iteration and thread
        const double flop = (double)grid * kThreads * (double)iters * 4.0 * kChains * 2.0;
        *h_tflops = flop / (med * 1e-3) / 1e12;
        if (h_ms) *h_ms = med;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
