// Synthetic sphere frames on the GPU (Sec. 5 evaluates the detector on
// frames of 100 rendered spheres with Poisson and Gaussian noise; the paper
// names no shading model).
//
// Reading: each sphere is an optically thin fluorescent droplet, so a pixel's
// brightness is proportional to the chord length through the sphere,
// sqrt(1 - d^2 / R^2) at distance d from the centre, averaged over ss x ss
// sub-pixel samples (pixel centres at integer coordinates); the frame is a
// background plus the spheres' contributions in table order, every step an
// explicitly rounded single-precision operation.  Counts are
//   floor(lambda + sqrt(lambda) z1 + read_noise z2 + 1/2) clipped to [0, 4095],
//   lambda = gain * intensity, in double,
// with z1, z2 sums of twelve uniforms minus 6; the uniforms are the top 24
// bits of Philox4x32-10 blocks (Salmon et al., SC'11), counter (pixel index
// low, high, draw, 0), key (seed low, high), three blocks per normal.
//
// A CTA renders a 16 x 16 tile: it first lists, in table order, the spheres
// whose disc (plus one pixel) meets the tile; spheres left out contribute
// exactly zero to every sample of the tile, so the sums are unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dog.h"

namespace {

constexpr int RT = 16;                 // tile edge
constexpr int RTHREADS = RT * RT;
constexpr int MAX_SPHERES = 8192;      // shared-memory list of one tile

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Sum of twelve uniforms minus 6 (exact in double: multiples of 2^-24 below 12).
__device__ double normal12(unsigned long long pix, uint32_t draw0, uint32_t k0, uint32_t k1) {
    double s = 0.0;
    for (uint32_t b = 0; b < 3; ++b) {
        uint32_t c[4] = {(uint32_t)pix, (uint32_t)(pix >> 32), draw0 + b, 0u};
        philox4x32_10(c, k0, k1);
#pragma unroll
        for (int q = 0; q < 4; ++q) s = __dadd_rn(s, __dmul_rn((double)(c[q] >> 8), 1.0 / 16777216.0));
    }
    return __dsub_rn(s, 6.0);
}

__global__ void __launch_bounds__(RTHREADS) render_spheres_kernel(const float4* __restrict__ sph, int S, int H,
                                                                  int W, int ss, float bg, double gain,
                                                                  double read_noise, uint32_t k0, uint32_t k1,
                                                                  float* inten, uint16_t* counts, int pitch) {
    __shared__ int list[MAX_SPHERES];
    __shared__ int wsum[RTHREADS / 32];
    __shared__ int n_list;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * RT, y0 = blockIdx.y * RT;
    const float tx0 = (float)x0 - 0.5f, tx1 = (float)(x0 + RT) - 0.5f;
    const float ty0 = (float)y0 - 0.5f, ty1 = (float)(y0 + RT) - 0.5f;
    if (tid == 0) n_list = 0;
    __syncthreads();
    // spheres meeting the tile, in table order (chunks of RTHREADS, block scan)
    for (int base = 0; base < S; base += RTHREADS) {
        const int s = base + tid;
        int keep = 0;
        if (s < S) {
            const float4 q = sph[s];
            const float m = q.z + 1.0f;
            keep = (q.x + m >= tx0 && q.x - m <= tx1 && q.y + m >= ty0 && q.y - m <= ty1) ? 1 : 0;
        }
        int incl = keep;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < RTHREADS / 32; ++w) {
            before += (w < warp) ? wsum[w] : 0;
            total += wsum[w];
        }
        if (keep) list[n_list + before + incl - 1] = s;
        __syncthreads();
        if (tid == 0) n_list += total;
        __syncthreads();
    }
    const int x = x0 + (tid % RT), y = y0 + (tid / RT);
    if (x >= W || y >= H) return;
    const float inv_n = 1.0f / (float)(ss * ss);
    float I = bg;
    const int n = n_list;
    for (int t = 0; t < n; ++t) {
        const float4 q = sph[list[t]];
        const float inv_r2 = __fdiv_rn(1.0f, __fmul_rn(q.z, q.z));
        float acc = 0.0f;
        for (int j = 0; j < ss; ++j) {
            const float v = __fadd_rn((float)y, __fsub_rn(__fdiv_rn((float)(2 * j + 1), (float)(2 * ss)), 0.5f));
            const float dy = __fsub_rn(v, q.y);
            const float dy2 = __fmul_rn(dy, dy);
            for (int i = 0; i < ss; ++i) {
                const float u = __fadd_rn((float)x, __fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)(2 * ss)), 0.5f));
                const float dx = __fsub_rn(u, q.x);
                const float qq = __fsub_rn(1.0f, __fmul_rn(__fadd_rn(__fmul_rn(dx, dx), dy2), inv_r2));
                if (qq > 0.0f) acc = __fadd_rn(acc, __fsqrt_rn(qq));
            }
        }
        I = __fadd_rn(I, __fmul_rn(q.w, __fmul_rn(acc, inv_n)));
    }
    if (inten) inten[(size_t)y * W + x] = I;
    const unsigned long long pix = (unsigned long long)y * (unsigned long long)W + (unsigned long long)x;
    const double lam = __dmul_rn(gain, (double)I);
    const double z1 = normal12(pix, 0u, k0, k1), z2 = normal12(pix, 3u, k0, k1);
    const double sl = __dsqrt_rn(lam > 0.0 ? lam : 0.0);
    double v = floor(__dadd_rn(__dadd_rn(__dadd_rn(lam, __dmul_rn(sl, z1)), __dmul_rn(read_noise, z2)), 0.5));
    v = v < 0.0 ? 0.0 : (v > 4095.0 ? 4095.0 : v);
    counts[(size_t)y * pitch + x] = (uint16_t)v;
}

}  // namespace

extern "C" int dog_render_spheres(const float* d_spheres, int32_t n_spheres, int32_t img_h, int32_t img_w,
                                  int32_t ss, float background, double gain, double read_noise, uint64_t seed,
                                  float* d_intensity, uint16_t* d_counts, int32_t pitch, void* stream) {
    if ((n_spheres > 0 && !d_spheres) || n_spheres < 0 || !d_counts || img_h < 1 || img_w < 1 || pitch < img_w)
        return DOG_ERR_INVALID;
    if (!(ss == 1 || ss == 2 || ss == 4 || ss == 8)) return DOG_ERR_INVALID;
    if (n_spheres > MAX_SPHERES) return DOG_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(d_spheres) & 15) != 0) return DOG_ERR_INVALID;
    const dim3 grid((img_w + RT - 1) / RT, (img_h + RT - 1) / RT);
    if (grid.y > 65535) return DOG_ERR_UNSUPPORTED;
    render_spheres_kernel<<<grid, RTHREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4*>(d_spheres), n_spheres, img_h, img_w, ss, background, gain, read_noise,
        (uint32_t)seed, (uint32_t)(seed >> 32), d_intensity, d_counts, pitch);
    return cudaGetLastError() == cudaSuccess ? DOG_OK : DOG_ERR_CUDA;
}
