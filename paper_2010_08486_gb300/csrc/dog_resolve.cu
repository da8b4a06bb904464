// Strip-edge resolve (sm_103a): settles the candidates the fused detection
// kernel queued because their 3x3x3 neighbourhood crosses into the adjacent
// 32-column strip (Sec. 4: the maximum test over x, y and scale).
#include <cuda_runtime.h>

#include <atomic>

#include "dog_internal.cuh"
#include "dog_device.cuh"

namespace dogk {

// ---------------------------------------------------------------------------
// Resolve: one CTA per queued strip-edge candidate (grid-stride).  The D
// values of the neighbouring strip's edge column xn are recomputed with the
// fused kernel's exact operation order (horizontal then vertical FMA chains
// from zero in ascending tap order, then c * (a - b)), so they equal what that
// strip held.  The candidate needs L_m at rows y-1 .. y+1 for the levels
// m = l-1 .. l+2; the image patch those chains read (rows y-1-Rc .. y+1+Rc,
// columns xn-Rc .. xn+Rc, reflected; Rc the largest of the four radii) is
// staged in shared memory once, the horizontal chains of all four levels run
// one per thread, and twelve threads run the vertical chains.
constexpr int RES_THREADS = 256;

__host__ __device__ inline int resolve_smem_floats(int R) {
    return (2 * R + 3) * (2 * R + 1) + 4 * (2 * R + 3) + 4 * (2 * R + 1) + 16;
}

// Eight CTAs per SM (the launch's grid cap): 32 registers per thread.
__global__ void __launch_bounds__(RES_THREADS, 8) dog_resolve_kernel(const __grid_constant__ ResolveParams p) {
    extern __shared__ float rsm[];
    const int tid = threadIdx.x;
    const int npend = min(*p.pend_count, p.pend_cap);
    for (int q = blockIdx.x; q < npend; q += gridDim.x) {
        const Pending e = p.pend[q];
        const void* img = p.img;
        int dtype = p.dtype, H = p.H, W = p.W, pitch = p.pitch;
        dog_blob* blobs = p.blobs;
        int* count = p.count;
        if (p.frames) {
            const FrameDesc f = p.frames[e.frame];
            img = f.img; dtype = f.dtype; H = f.h; W = f.w; pitch = f.pitch;
            blobs = p.blobs + f.blob_off;
            count = p.count + e.frame;
        }
        const int st_lo = dtype == DTYPE_U16_STRETCH ? p.lohi[2 * e.frame] : 0;
        const int st_hi = dtype == DTYPE_U16_STRETCH ? p.lohi[2 * e.frame + 1] : 0;
        const float st_rcp = stretch_rcp(st_lo, st_hi);
        const int lx = e.x % TX;
        const int xn = (lx == 0) ? e.x - 1 : e.x + 1;   // the column held by the other strip
        const int l = e.level;
        const int m0 = max(l - 1, 0), m1 = min(l + 2, p.K - 1);   // levels m0 .. m1
        const int nm = m1 - m0 + 1;
        // radii of the (up to) four levels and the prefix offsets of their
        // horizontal chains, in named scalars (no dynamically indexed arrays)
        const int ra = p.r[m0];
        const int rb = nm > 1 ? p.r[m0 + 1] : 0;
        const int rc = nm > 2 ? p.r[m0 + 2] : 0;
        const int rd = nm > 3 ? p.r[m0 + 3] : 0;
        const int Rc = max(max(ra, rb), max(rc, rd));
        const int o1 = 2 * ra + 3;
        const int o2 = o1 + (nm > 1 ? 2 * rb + 3 : 0);
        const int o3 = o2 + (nm > 2 ? 2 * rc + 3 : 0);
        const int o4 = o3 + (nm > 3 ? 2 * rd + 3 : 0);
        const int pw = 2 * Rc + 1, ph = 2 * Rc + 3;
        float* patch = rsm;                      // ph x pw
        float* hb = rsm + ph * pw;               // 4 x ph: horizontal sums per level
        float* wsm = hb + 4 * ph;                // 4 x pw: taps of the four levels
        float* Lv = wsm + 4 * pw;                // 4 x 3
        // taps
        for (int i = tid; i < 4 * pw; i += RES_THREADS) {
            const int mi = i / pw, t = i - mi * pw;
            const int r = mi == 0 ? ra : (mi == 1 ? rb : (mi == 2 ? rc : rd));
            wsm[i] = (mi < nm && t <= 2 * r) ? __ldg(p.w + p.woff[m0 + mi] + t) : 0.0f;
        }
        // patch: thread (row phase jt, column cc); rows jt, jt + rpp, ...; the
        // loads of four rows are issued before any is converted
        {
            const int rpp = RES_THREADS / pw;
            const int jt = tid / pw, cc = tid - jt * pw;
            if (jt < rpp) {
                const int xr = refl(xn - Rc + cc, W);
                const int y0 = e.y - 1 - Rc;
                for (int j = jt; j < ph; j += 4 * rpp) {
                    unsigned v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int jj = j + u * rpp;
                        v[u] = jj < ph ? load_raw(img, dtype, pitch, refl(y0 + jj, H), xr) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int jj = j + u * rpp;
                        if (jj < ph) patch[jj * pw + cc] = raw_to_px(v[u], dtype, st_lo, st_hi, st_rcp);
                    }
                }
            }
        }
        __syncthreads();
        // horizontal chains: level mi, patch rows Rc - r .. Rc + 2 + r
        for (int it = tid; it < o4; it += RES_THREADS) {
            const int mi = (it >= o1) + (it >= o2) + (it >= o3);
            const int j = it - (mi == 0 ? 0 : (mi == 1 ? o1 : (mi == 2 ? o2 : o3)));
            const int r = mi == 0 ? ra : (mi == 1 ? rb : (mi == 2 ? rc : rd));
            const float* w = wsm + mi * pw;
            const float* src = patch + (Rc - r + j) * pw + (Rc - r);
            float acc = 0.0f;
#pragma unroll 8
            for (int t = 0; t <= 2 * r; ++t) acc = __fmaf_rn(w[t], src[t], acc);
            hb[mi * ph + j] = acc;
        }
        __syncthreads();
        if (tid < 3 * nm) {
            const int mi = tid / 3, yi = tid - 3 * mi;
            const int r = mi == 0 ? ra : (mi == 1 ? rb : (mi == 2 ? rc : rd));
            const float* w = wsm + mi * pw;
            const float* src = hb + mi * ph + yi;
            float acc = 0.0f;
#pragma unroll 8
            for (int t = 0; t <= 2 * r; ++t) acc = __fmaf_rn(w[t], src[t], acc);
            Lv[mi * 3 + yi] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            bool keep = true;
            for (int ll = max(l - 1, 0); ll <= min(l + 1, p.P - 1); ++ll) {
                for (int yi = 0; yi < 3; ++yi) {
                    const int y = e.y - 1 + yi;
                    if (y < 0 || y >= H) continue;
                    const float d = __fmul_rn(__ldg(p.c + ll), __fsub_rn(Lv[(ll - m0) * 3 + yi], Lv[(ll + 1 - m0) * 3 + yi]));
                    if (d > e.response) keep = false;
                }
            }
            if (keep) {
                const int idx = atomicAdd(count, 1);
                if (idx < p.cap) {
                    dog_blob bl;
                    bl.x = e.x; bl.y = e.y; bl.level = l; bl.sigma = __ldg(p.c + p.P + l); bl.response = e.response;
                    blobs[idx] = bl;
                } else {
                    atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                }
            }
        }
        __syncthreads();   // the patch is rewritten by the next candidate
    }
}

// Raised once per device; atomic because several host threads may launch.
static std::atomic<int> g_resolve_smem[64];

cudaError_t launch_resolve(const ResolveParams& p, int max_pending, cudaStream_t s) {
    int R = 0;
    for (int m = 0; m < p.K; ++m) R = p.r[m] > R ? p.r[m] : R;
    const int smem = (int)sizeof(float) * resolve_smem_floats(R);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::atomic<int>& lim = g_resolve_smem[dev & 63];
    if (smem > 48 * 1024 && lim.load(std::memory_order_acquire) < smem) {
        e = cudaFuncSetAttribute(dog_resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int cur = lim.load(std::memory_order_relaxed);
        while (cur < smem && !lim.compare_exchange_weak(cur, smem)) {
        }
    }
    int grid = max_pending;
    if (grid < 1) grid = 1;
    if (grid > 152 * 8) grid = 152 * 8;
    dog_resolve_kernel<<<grid, RES_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace dogk
