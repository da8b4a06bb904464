// Contrast stretch of 12-bit frames (Sec. 4: the optional first step maps a
// frame to [0, 1] with 0.35% saturation; Table 2 shows it dominating the
// paper's CPU preprocessing).
//
// Reading: with the frame's n counts sorted ascending and k = floor(sat/2 n),
// the count at rank k maps to 0, the count at rank n-1-k maps to 1, and the
// map (c - lo) / (hi - lo) is clipped to [0, 1]; counts above 4095 count as
// 4095.  On the GPU the order statistics come from a 4096-bin histogram per
// frame (shared-memory counts, one global atomic per nonzero bin and CTA) and
// a block-wide scan of it; the map itself is applied where the detection
// kernels ingest the frame (stretch_px) or by stretch_apply_kernel.
#include <cuda_runtime.h>

#include <cmath>

#include "dog_internal.cuh"
#include "dog_device.cuh"

namespace dogk {

constexpr int HIST_THREADS = 256;
constexpr int LIM_THREADS = 1024;
static_assert(STRETCH_BINS == 4 * LIM_THREADS, "four bins per thread in the limits scan");

// Histogram of frame blockIdx.y; CTAs blockIdx.x take rows blockIdx.x,
// blockIdx.x + gridDim.x, ...  frames == nullptr: the single frame (img, H, W,
// pitch).  hist: STRETCH_BINS counts per frame, zeroed by the caller.
__global__ void __launch_bounds__(HIST_THREADS) stretch_hist_kernel(const dog_frame* frames, const uint16_t* img,
                                                                    int H, int W, int pitch, int* hist) {
    __shared__ int sh[STRETCH_BINS];
    const int f = blockIdx.y;
    if (frames) {
        const dog_frame fr = frames[f];
        if (fr.dtype != DOG_DTYPE_U16) return;   // only 12-bit frames are stretched
        img = static_cast<const uint16_t*>(fr.ptr);
        H = fr.h;
        W = fr.w;
        pitch = fr.pitch;
    }
    for (int q = threadIdx.x; q < STRETCH_BINS; q += HIST_THREADS) sh[q] = 0;
    __syncthreads();
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const uint16_t* row = img + (size_t)y * pitch;
        for (int x = threadIdx.x; x < W; x += HIST_THREADS) {
            const int v = min((int)__ldg(row + x), STRETCH_BINS - 1);
            atomicAdd(&sh[v], 1);
        }
    }
    __syncthreads();
    int* out = hist + (size_t)f * STRETCH_BINS;
    for (int q = threadIdx.x; q < STRETCH_BINS; q += HIST_THREADS)
        if (sh[q]) atomicAdd(&out[q], sh[q]);
}

// Limits of frame blockIdx.x from its histogram: the counts at ranks k and
// n-1-k (k = floor(sat/2 n), at most (n-1)/2): the bin v with
// #(c < v) <= rank < #(c <= v).  lohi[2f] = lo, lohi[2f+1] = hi.
__global__ void __launch_bounds__(LIM_THREADS) stretch_limits_kernel(const dog_frame* frames, int H, int W,
                                                                     double sat, const int* hist, int* lohi) {
    __shared__ int wsum[LIM_THREADS / 32];
    const int f = blockIdx.x;
    if (frames) {
        const dog_frame fr = frames[f];
        if (fr.dtype != DOG_DTYPE_U16) return;
        H = fr.h;
        W = fr.w;
    }
    const long long n = (long long)H * W;
    long long k = (long long)floor(sat * 0.5 * (double)n);
    if (k > (n - 1) / 2) k = (n - 1) / 2;
    const long long r_lo = k, r_hi = n - 1 - k;
    const int* h = hist + (size_t)f * STRETCH_BINS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int c[4];
    int tsum = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        c[u] = h[4 * tid + u];
        tsum += c[u];
    }
    // block exclusive scan of the per-thread sums
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    long long below = (long long)(incl - tsum) + (warp > 0 ? wsum[warp - 1] : 0);   // #(c < 4 tid)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long long upto = below + c[u];   // #(c <= v)
        const int v = 4 * tid + u;
        if (below <= r_lo && r_lo < upto) lohi[2 * f] = v;
        if (below <= r_hi && r_hi < upto) lohi[2 * f + 1] = v;
        below = upto;
    }
}

// The stretched frame (FP32, [0, 1]) of one 12-bit frame with limits lohi.
// Row blockIdx.y (grid-strided); each thread maps 4 consecutive pixels, with
// one 8-byte load and one 16-byte store when both rows allow it.
__global__ void __launch_bounds__(256) stretch_apply_kernel(const uint16_t* img, int H, int W, int pitch,
                                                            const int* lohi, float* out, int out_pitch) {
    const int lo = lohi[0], hi = lohi[1];
    const float rcp = stretch_rcp(lo, hi);
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const uint16_t* src = img + (size_t)y * pitch;
        float* dst = out + (size_t)y * out_pitch;
        const bool vec = ((reinterpret_cast<size_t>(src) & 7) == 0) && ((reinterpret_cast<size_t>(dst) & 15) == 0);
        for (int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x); x < W; x += 4 * gridDim.x * blockDim.x) {
            if (vec && x + 4 <= W) {
                const uint2 v = __ldg(reinterpret_cast<const uint2*>(src + x));
                *reinterpret_cast<float4*>(dst + x) =
                    make_float4(stretch_px(v.x & 0xffffu, lo, hi, rcp), stretch_px(v.x >> 16, lo, hi, rcp),
                                stretch_px(v.y & 0xffffu, lo, hi, rcp), stretch_px(v.y >> 16, lo, hi, rcp));
            } else {
                for (int u = x; u < x + 4 && u < W; ++u) dst[u] = stretch_px(__ldg(src + u), lo, hi, rcp);
            }
        }
    }
}

cudaError_t launch_stretch_limits(const dog_frame* frames, int n, const uint16_t* img, int H, int W, int pitch,
                                  double sat, int num_sms, int* hist, int* lohi, cudaStream_t s) {
    if (n < 1 || n > 65535) return cudaErrorInvalidValue;   // frames index the grid's y dimension
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * STRETCH_BINS * (size_t)n, s);
    if (e != cudaSuccess) return e;
    // about two CTAs per SM over the whole call; a frame's CTAs split its rows
    int per = (2 * num_sms + n - 1) / n;
    if (per < 1) per = 1;
    if (!frames && per > H) per = H;
    if (per > 1024) per = 1024;
    stretch_hist_kernel<<<dim3(per, n), HIST_THREADS, 0, s>>>(frames, img, H, W, pitch, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stretch_limits_kernel<<<n, LIM_THREADS, 0, s>>>(frames, H, W, sat, hist, lohi);
    return cudaGetLastError();
}

cudaError_t launch_stretch_apply(const uint16_t* img, int H, int W, int pitch, const int* lohi, float* out,
                                 int out_pitch, int num_sms, cudaStream_t s) {
    const int gx = (W + 4 * 256 - 1) / (4 * 256);
    int gy = (8 * num_sms + gx - 1) / gx;
    if (gy > H) gy = H;
    if (gy > 65535) gy = 65535;
    stretch_apply_kernel<<<dim3(gx, gy), 256, 0, s>>>(img, H, W, pitch, lohi, out, out_pitch);
    return cudaGetLastError();
}

}  // namespace dogk

using namespace dogk;

extern "C" int dog_stretch_limits(const uint16_t* d_img, int32_t img_h, int32_t img_w, int32_t pitch, double sat,
                                  int32_t* d_hist, int32_t* d_lohi, void* stream) {
    if (!d_img || !d_hist || !d_lohi || img_h < 1 || img_w < 1 || pitch < img_w) return DOG_ERR_INVALID;
    if (!(sat >= 0.0 && sat < 1.0)) return DOG_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DOG_ERR_CUDA;
    return launch_stretch_limits(nullptr, 1, d_img, img_h, img_w, pitch, sat, sms, d_hist, d_lohi,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? DOG_OK
               : DOG_ERR_CUDA;
}

extern "C" int dog_stretch(const uint16_t* d_img, int32_t img_h, int32_t img_w, int32_t pitch,
                           const int32_t* d_lohi, float* d_out, int32_t out_pitch, void* stream) {
    if (!d_img || !d_lohi || !d_out || img_h < 1 || img_w < 1 || pitch < img_w || out_pitch < img_w)
        return DOG_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DOG_ERR_CUDA;
    return launch_stretch_apply(d_img, img_h, img_w, pitch, d_lohi, d_out, out_pitch, sms,
                                static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? DOG_OK
               : DOG_ERR_CUDA;
}
