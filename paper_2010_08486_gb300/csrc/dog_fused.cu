// Fused DoG detector kernel: the 12-producer-warp forms, the launcher that
// picks a form, and the batched set-up kernel.  The kernel itself is in
// dog_fused_forms.cuh.
#include "dog_fused_forms.cuh"

namespace dogk {

cudaError_t launch_fused_w8(const FusedParams& p, int grid, cudaStream_t s);   // dog_fused_w8.cu

cudaError_t launch_fused(const FusedParams& p, int grid, cudaStream_t s) {
    if (p.P < 1 || p.P > MAX_LEVELS - 1) return cudaErrorInvalidValue;
    if (p.nw == 8) return launch_fused_w8(p, grid, s);
    if (p.nw == 12) return launch_fused_form<12>(p, grid, s);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Batched set-up: per-frame descriptors and the exclusive prefix sum of tiles
// (strips x row bands) that the persistent kernel walks.  One CTA.  The
// frames whose tiles make up the last `tail_tiles` of the walk are cut into
// four times as many row bands, so the persistent CTAs run out of work at
// about the same time instead of leaving most of them idle in a last,
// partly filled round of whole tiles.

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the exclusive prefix and adds the block total to *carry.
__device__ __forceinline__ long long block_scan(long long v, long long* wsum, long long* carry) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    const long long incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    const long long excl = *carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) *carry += incl;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(1024) dog_batch_prep_kernel(const dog_frame* frames, int n, int band,
                                                              int tail_tiles, int blob_cap, bool stretch,
                                                              FrameDesc* desc,
                                                              long long* cand_off, long long* out_off,
                                                              int* hw, long long* ntiles) {
    __shared__ long long carry, total;
    __shared__ long long wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    // pass 1: uniform bands
    for (int base = 0; base < n; base += blockDim.x) {
        const int f = base + threadIdx.x;
        long long tiles = 0;
        FrameDesc d{};
        if (f < n) {
            const dog_frame fr = frames[f];
            d.img = fr.ptr;
            d.h = fr.h;
            d.w = fr.w;
            d.pitch = fr.pitch;
            d.dtype = (stretch && fr.dtype == DOG_DTYPE_U16) ? DTYPE_U16_STRETCH : fr.dtype;
            d.blob_off = (long long)f * blob_cap;
            d.n_strips = (fr.w + TX - 1) / TX;
            d.band = (band > 0 && band < fr.h) ? band : fr.h;
            d.n_bands = (fr.h + d.band - 1) / d.band;
            tiles = (long long)d.n_strips * d.n_bands;
            cand_off[f] = (long long)f * blob_cap;
            out_off[f] = fr.blob_off;
            hw[2 * f] = fr.h;
            hw[2 * f + 1] = fr.w;
        }
        const long long excl = block_scan(tiles, wsum, &carry);
        if (f < n) {
            d.tile_begin = excl;
            desc[f] = d;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) { total = carry; carry = 0; }
    __syncthreads();
    // pass 2: finer bands for the frames of the last tail_tiles tiles
    for (int base = 0; base < n; base += blockDim.x) {
        const int f = base + threadIdx.x;
        long long tiles = 0;
        FrameDesc d{};
        if (f < n) {
            d = desc[f];
            if (tail_tiles > 0 && d.tile_begin + (long long)d.n_strips * d.n_bands > total - tail_tiles) {
                const int b4 = ((d.band + 3) / 4 + MB - 1) / MB * MB;
                d.band = b4 > 0 ? b4 : MB;
                d.n_bands = (d.h + d.band - 1) / d.band;
            }
            tiles = (long long)d.n_strips * d.n_bands;
        }
        const long long excl = block_scan(tiles, wsum, &carry);
        if (f < n) {
            d.tile_begin = excl;
            desc[f] = d;
        }
    }
    if (threadIdx.x == 0) *ntiles = carry;
}

cudaError_t launch_batch_prep(const dog_frame* frames, int n, int band, int tail_tiles, int blob_cap,
                              bool stretch, FrameDesc* desc, long long* cand_off, long long* out_off, int* hw,
                              long long* ntiles, cudaStream_t s) {
    dog_batch_prep_kernel<<<1, 1024, 0, s>>>(frames, n, band, tail_tiles, blob_cap, stretch, desc, cand_off,
                                             out_off, hw, ntiles);
    return cudaGetLastError();
}

}  // namespace dogk
