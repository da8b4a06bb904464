// Fused DoG detector kernel for sm_103a.
//
// Method (arXiv 2010.08486): scale space L_i = g(sigma_i) * I (Sec. 3), DoG
// D_i = c_i (L_i - L_{i+1}) (Eq. 2-3), voxels equal to their 3x3x3 maximum
// and above the threshold (Sec. 4, Sec. 4.1).
//
// Design.  A CTA owns a strip of TX = 32 output columns and walks down a
// band of rows in blocks of MB = 8 rows, so every input pixel of the strip
// is read once from global memory for all K scales and no vertical halo is
// recomputed.  Each of the eight warps owns a fixed set of levels, chosen on
// the host to balance taps.  For each block and owned level a warp
//   1. runs the horizontal pass of the next 8 input rows into the level's
//      shared-memory ring (which runs ceil(2r/8) blocks ahead),
//   2. runs the vertical pass over the ring into the block's L rows,
//   3. shifts the ring up by 8 rows.
// Both passes are register-blocked 1-D correlations (8 outputs per lane,
// taps unrolled for radii <= RT_MAX), summing taps in ascending order with
// FMA from zero -- the resolve kernel below repeats the same order and so
// reproduces any value bit for bit.  Then all threads form D in place and
// test the previous block's rows against their 26 neighbours; survivors are
// compacted with one warp ballot and one atomic per warp.  Neighbours in the
// adjacent strip are not held here: a candidate at a strip edge is queued and
// the resolve kernel recomputes the few D values it needs.
#include <cuda_runtime.h>

#include "dog_internal.cuh"

namespace dogk {

__device__ __forceinline__ int refl(int i, int n) {
    int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m >= n ? p - 1 - m : m;
}

__device__ __forceinline__ float load_px(const void* img, int dtype, int pitch, int y, int x) {
    if (dtype == DOG_DTYPE_U16) {
        unsigned short v = __ldg(reinterpret_cast<const unsigned short*>(img) + (size_t)y * pitch + x);
        return __fdiv_rn((float)v, 4095.0f);
    }
    return __ldg(reinterpret_cast<const float*>(img) + (size_t)y * pitch + x);
}

__device__ __forceinline__ float dog_value(float c, float a, float b) {
    return __fmul_rn(c, __fsub_rn(a, b));
}

// ---------------------------------------------------------------------------
// 1-D passes.  out[k] = sum_{t=0}^{2r} w[|t-r|] * in[k+t], k = 0..7, in
// ascending t, starting from 0.
template <int R>
__device__ __forceinline__ void hpass_t(const float* __restrict__ src, float* __restrict__ dst,
                                        const float* __restrict__ wsm) {
    float w[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) w[j] = wsm[j];
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
#pragma unroll
    for (int t = 0; t < 8 + 2 * R; ++t) {
        const float v = src[t];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int tap = t - k;
            if (tap >= 0 && tap <= 2 * R) {
                const int j = tap >= R ? tap - R : R - tap;
                acc[k] = __fmaf_rn(w[j], v, acc[k]);
            }
        }
    }
    float4* d4 = reinterpret_cast<float4*>(dst);
    d4[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    d4[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

template <int R>
__device__ __forceinline__ void vpass_t(const float* __restrict__ src, float* const* dst,
                                        const float* __restrict__ wsm) {
    float w[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) w[j] = wsm[j];
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
#pragma unroll
    for (int t = 0; t < 8 + 2 * R; ++t) {
        const float v = src[t * RING_STRIDE];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int tap = t - k;
            if (tap >= 0 && tap <= 2 * R) {
                const int j = tap >= R ? tap - R : R - tap;
                acc[k] = __fmaf_rn(w[j], v, acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) *dst[k] = acc[k];
}

// Radii above RT_MAX: same arithmetic order with a rolled tap loop.
__device__ __noinline__ void hpass_g(const float* __restrict__ src, float* __restrict__ dst,
                                     const float* __restrict__ wsm, int r) {
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
    for (int t = 0; t < 8 + 2 * r; ++t) {
        const float v = src[t];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int tap = t - k;
            if (tap >= 0 && tap <= 2 * r) {
                const int j = tap >= r ? tap - r : r - tap;
                acc[k] = __fmaf_rn(wsm[j], v, acc[k]);
            }
        }
    }
    float4* d4 = reinterpret_cast<float4*>(dst);
    d4[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    d4[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

__device__ __noinline__ void vpass_g(const float* __restrict__ src, float* const* dst,
                                     const float* __restrict__ wsm, int r) {
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
    for (int t = 0; t < 8 + 2 * r; ++t) {
        const float v = src[t * RING_STRIDE];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int tap = t - k;
            if (tap >= 0 && tap <= 2 * r) {
                const int j = tap >= r ? tap - r : r - tap;
                acc[k] = __fmaf_rn(wsm[j], v, acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) *dst[k] = acc[k];
}

#define DOG_CASES(X)                                                                      \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
    X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)  \
    X(31) X(32) X(33) X(34) X(35) X(36) X(37) X(38) X(39) X(40) X(41) X(42) X(43) X(44)  \
    X(45) X(46) X(47) X(48)

__device__ __forceinline__ void hpass(int r, const float* src, float* dst, const float* wsm) {
    switch (r) {
#define DOG_H(R) \
    case R: hpass_t<R>(src, dst, wsm); return;
        DOG_CASES(DOG_H)
#undef DOG_H
        default: hpass_g(src, dst, wsm, r); return;
    }
}

__device__ __forceinline__ void vpass(int r, const float* src, float* const* dst, const float* wsm) {
    switch (r) {
#define DOG_V(R) \
    case R: vpass_t<R>(src, dst, wsm); return;
        DOG_CASES(DOG_V)
#undef DOG_V
        default: vpass_g(src, dst, wsm, r); return;
    }
}

// ---------------------------------------------------------------------------
struct TileCtx {
    const void* img;
    int dtype, H, W, pitch;
    int frame;
    int x0, y0, y1;
    dog_blob* blobs;
    int* count;
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Shared scalars of one CTA (static shared memory).
struct SmemSmall {
    float c[MAX_LEVELS];
    float sig[MAX_LEVELS];
    float gk[MAX_LEVELS];     // sum_b gH_b kappa_b(t_l)
    float gdk[MAX_LEVELS];    // sum_b gH_b dkappa_b/dt(t_l)
    int kb[MAX_LEVELS][2];    // nonzero soft-histogram bins of each plane
    float kw[MAX_LEVELS][2];
    float soft[DOG_MAX_NBINS];
    float dc[MAX_LEVELS];
    float dt[MAX_LEVELS];
    int tile;
};

__device__ void process_tile(const FusedParams& p, float* sm, SmemSmall& ss, const TileCtx& tc) {
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int R = p.R;
    const int P = p.P;
    const int CIN = p.in_rows;        // power of two
    const int S = p.in_stride;
    const int ncols = TX + 2 * R;     // input columns per row
    const int yb0 = tc.y0 - 1;
    const int nblk = (tc.y1 - tc.y0 + 2 + MB - 1) / MB;
    int emax = 0;
    for (int i = 0; i < p.K; ++i) emax = max(emax, p.lv[i].e);
    const int yorg = yb0 - MB * emax;   // input-ring slot origin

    float* in = sm + p.in_off;
    float* dbuf = sm + p.d_off;

    // initial input rows: those read at block -emax
    {
        const int ya = yorg + p.dmin;
        const int yz = yorg + p.dmax + MB;
        const int n = (yz - ya) * ncols;
        for (int q = tid; q < n; q += NTHREADS) {
            const int yy = ya + q / ncols;
            const int cc = q % ncols;
            const float v = load_px(tc.img, tc.dtype, tc.pitch, refl(yy, tc.H), refl(tc.x0 - R + cc, tc.W));
            in[((yy - yorg) & (CIN - 1)) * S + cc] = v;
        }
    }
    __syncthreads();

    constexpr int PF = (MB * (TX + 2 * DOG_MAX_RADIUS) + NTHREADS - 1) / NTHREADS;
    const int npf = MB * ncols;

    for (int b = -emax; b < nblk; ++b) {
        const int yb = yb0 + MB * b;
        // prefetch the rows block b+1 adds (latency hidden behind phase A)
        float pf[PF];
        const int ynew = yorg + MB * (b + emax + 1) + p.dmax;
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int q = tid + j * NTHREADS;
            pf[j] = 0.0f;
            if (q < npf && b + 1 < nblk) {
                const int yy = ynew + q / ncols;
                const int cc = q % ncols;
                pf[j] = load_px(tc.img, tc.dtype, tc.pitch, refl(yy, tc.H), refl(tc.x0 - R + cc, tc.W));
            }
        }

        // ---- phase A: horizontal + vertical passes of this warp's levels
        const int nl = p.warp_nlev[warp];
        for (int li = 0; li < nl; ++li) {
            const int i = p.warp_lev[warp][li];
            const LevelInfo L = p.lv[i];
            const int c = b + L.e;
            if (c < 0) continue;
            float* ring = sm + L.ring_off;
            const float* wsm = sm + p.w_off + L.woff;
            {
                const int rho = lane >> 2, g = lane & 3;
                const int yy = yb + L.delta + rho;     // input row of this lane
                const float* src = in + ((yy - yorg) & (CIN - 1)) * S + (R - L.r) + 8 * g;
                float* dst = ring + (L.ring_rows - MB + rho) * RING_STRIDE + 8 * g;
                hpass(L.r, src, dst, wsm);
            }
            __syncwarp();
            if (b >= 0) {
                float* dst[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    dst[k] = dbuf + (i * DSLOTS + (MB * b + k + 2) % DSLOTS) * TX + lane;
                vpass(L.r, ring + lane, dst, wsm);
            }
            __syncwarp();
            {
                // shift the ring up by MB rows; each (row, quad) moves within one lane
                float4* r4 = reinterpret_cast<float4*>(ring);
                const int rows = L.ring_rows - MB;
                const int c4 = lane & 7;
                for (int row = lane >> 3; row < rows; row += 4)
                    r4[row * (RING_STRIDE / 4) + c4] = r4[(row + MB) * (RING_STRIDE / 4) + c4];
            }
            __syncwarp();
        }
        __syncthreads();

        // ---- phase B: D_i = c_i (L_i - L_{i+1}) in place for rows yb..yb+7
        if (b >= 0) {
            const int k = warp;
            const int x = lane;
            const int y = yb + k;
            const int slot = (MB * b + k + 2) % DSLOTS;
            float* col = dbuf + slot * TX + x;
            float Lnext = col[0];
            for (int i = 0; i < P; ++i) {
                const float Li = Lnext;
                Lnext = col[(i + 1) * DSLOTS * TX];
                const float d = dog_value(ss.c[i], Li, Lnext);
                col[i * DSLOTS * TX] = d;
                if (p.mode == MODE_DUMP && y >= tc.y0 && y < tc.y1 && tc.x0 + x < tc.W)
                    p.dump[((size_t)i * tc.H + y) * tc.W + tc.x0 + x] = d;
            }
        }
        // store the prefetched input rows (slots not read by this or the next block's old rows)
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int q = tid + j * NTHREADS;
            if (q < npf && b + 1 < nblk) {
                const int yy = ynew + q / ncols;
                in[((yy - yorg) & (CIN - 1)) * S + q % ncols] = pf[j];
            }
        }
        __syncthreads();

        // ---- phase C: test row yb-1+warp against its 26 neighbours
        if (b >= 0 && p.mode != MODE_DUMP) {
            const int y = yb - 1 + warp;
            const bool row_ok = (y >= tc.y0 && y < tc.y1);
            const int x = lane;
            const int gx = tc.x0 + x;
            const bool col_ok = gx < tc.W;
            const int sc = (MB * b + warp + 1) % DSLOTS;    // slot of row y
            const int sm1 = (MB * b + warp) % DSLOTS;       // row y-1
            const int sp1 = (MB * b + warp + 2) % DSLOTS;   // row y+1
            const bool ym_ok = y - 1 >= 0, yp_ok = y + 1 < tc.H;
            const bool left_out = (x == 0 && tc.x0 > 0);
            const bool right_out = (x == TX - 1 && gx + 1 < tc.W);
            const bool soft = (p.mode == MODE_SOFT || p.mode == MODE_BWD);
            float Gprev = 0.0f;
            for (int l = 0; l < P; ++l) {
                const float d = dbuf[(l * DSLOTS + sc) * TX + x];
                bool cand = row_ok && col_ok && (soft || d > p.thr);
                bool edge = false;
                if (__any_sync(0xffffffffu, cand)) {
                    if (cand) {
#pragma unroll 1
                        for (int dl = -1; dl <= 1 && cand; ++dl) {
                            const int ll = l + dl;
                            if (ll < 0 || ll >= P) continue;
#pragma unroll
                            for (int dy = -1; dy <= 1; ++dy) {
                                if ((dy < 0 && !ym_ok) || (dy > 0 && !yp_ok)) continue;
                                const int s = dy < 0 ? sm1 : (dy > 0 ? sp1 : sc);
                                const float* row = dbuf + (ll * DSLOTS + s) * TX;
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    if (dl == 0 && dy == 0 && dx == 0) continue;
                                    const int xx = x + dx;
                                    if (xx < 0) { edge |= left_out; continue; }
                                    if (xx >= TX) { edge |= right_out; continue; }
                                    if (tc.x0 + xx >= tc.W) continue;
                                    if (row[xx] > d) cand = false;
                                }
                            }
                        }
                    }
                }
                const bool direct = cand && !edge;
                const bool pend = cand && edge;
                if (p.mode == MODE_CANDIDATES) {
                    const unsigned m = __ballot_sync(0xffffffffu, direct);
                    if (m) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(tc.count, __popc(m));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (direct) {
                            const int idx = base + __popc(m & lanemask_lt());
                            if (idx < p.cap) {
                                dog_blob bl;
                                bl.x = gx; bl.y = y; bl.level = l; bl.sigma = ss.sig[l]; bl.response = d;
                                tc.blobs[idx] = bl;
                            } else {
                                atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                            }
                        }
                    }
                } else if (direct) {
                    const float s = 1.0f / (1.0f + __expf(-(d - p.thr) * p.inv_T));
                    if (p.mode == MODE_SOFT) {
                        atomicAdd(&ss.soft[ss.kb[l][0]], s * ss.kw[l][0]);
                        atomicAdd(&ss.soft[ss.kb[l][1]], s * ss.kw[l][1]);
                    } else {
                        const float G = ss.gk[l] * s * (1.0f - s) * p.inv_T;
                        atomicAdd(&ss.dc[l], G * d / ss.c[l]);
                        atomicAdd(&ss.dt[l], s * ss.gdk[l]);
                    }
                }
                if (p.mode == MODE_BWD) {
                    float G = 0.0f;
                    if (direct) {
                        const float s = 1.0f / (1.0f + __expf(-(d - p.thr) * p.inv_T));
                        G = ss.gk[l] * s * (1.0f - s) * p.inv_T;
                    }
                    if (row_ok && col_ok) {
                        const float a = ss.c[l] * G - (l > 0 ? ss.c[l - 1] * Gprev : 0.0f);
                        p.A[((size_t)l * tc.H + y) * tc.W + gx] = a;
                        if (l == P - 1) p.A[((size_t)(l + 1) * tc.H + y) * tc.W + gx] = -ss.c[l] * G;
                    }
                    Gprev = G;
                }
                const unsigned mp = __ballot_sync(0xffffffffu, pend);
                if (mp) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(p.pend_count, __popc(mp));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (pend) {
                        const int idx = base + __popc(mp & lanemask_lt());
                        if (idx < p.pend_cap) {
                            Pending e;
                            e.frame = tc.frame; e.x = gx; e.y = y; e.level = l; e.response = d;
                            p.pend[idx] = e;
                        } else {
                            atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <bool BATCHED>
__global__ void __launch_bounds__(NTHREADS, 1) dog_fused_kernel(const __grid_constant__ FusedParams p) {
    extern __shared__ float4 dyn4[];
    float* sm = reinterpret_cast<float*>(dyn4);
    __shared__ SmemSmall ss;
    const int tid = threadIdx.x;
    for (int q = tid; q < p.w_total; q += NTHREADS) sm[p.w_off + q] = p.w[q];
    for (int q = tid; q < p.P; q += NTHREADS) ss.c[q] = p.c[q];
    for (int q = tid; q < p.P; q += NTHREADS) ss.sig[q] = 0.0f;
    if (p.mode == MODE_SOFT || p.mode == MODE_BWD) {
        for (int q = tid; q < p.nbins; q += NTHREADS) ss.soft[q] = 0.0f;
        for (int l = tid; l < p.P; l += NTHREADS) {
            float gk = 0.0f, gdk = 0.0f;
            int nb = 0;
            ss.kb[l][0] = 0; ss.kb[l][1] = 0; ss.kw[l][0] = 0.0f; ss.kw[l][1] = 0.0f;
            for (int b = 0; b < p.nbins; ++b) {
                const float k = p.kappa[l * p.nbins + b];
                if (p.gH) {
                    gk += p.gH[b] * k;
                    gdk += p.gH[b] * p.dkappa[l * p.nbins + b];
                }
                if (k != 0.0f && nb < 2) { ss.kb[l][nb] = b; ss.kw[l][nb] = k; ++nb; }
            }
            ss.gk[l] = gk; ss.gdk[l] = gdk; ss.dc[l] = 0.0f; ss.dt[l] = 0.0f;
        }
    }
    __syncthreads();

    if (!BATCHED) {
        // single frame: blockIdx.x enumerates (strip, band)
        if (p.mode == MODE_CANDIDATES) {
            for (int q = tid; q < p.P; q += NTHREADS) ss.sig[q] = p.c[p.P + q];
        }
        __syncthreads();
        TileCtx tc;
        tc.img = p.img; tc.dtype = p.dtype; tc.H = p.H; tc.W = p.W; tc.pitch = p.pitch; tc.frame = 0;
        const int strip = blockIdx.x % p.n_strips;
        const int band = blockIdx.x / p.n_strips;
        tc.x0 = strip * TX;
        tc.y0 = band * p.band;
        tc.y1 = min(p.H, tc.y0 + p.band);
        tc.blobs = p.blobs;
        tc.count = p.count;
        process_tile(p, sm, ss, tc);
    } else {
        for (int q = tid; q < p.P; q += NTHREADS) ss.sig[q] = p.c[p.P + q];
        const long long n_tiles = p.ntiles_dev ? *p.ntiles_dev : p.n_tiles;
        for (;;) {
            __syncthreads();
            if (tid == 0) ss.tile = atomicAdd(p.tile_counter, 1);
            __syncthreads();
            const long long t = ss.tile;
            if (t >= n_tiles) break;
            int lo = 0, hi = p.n_frames - 1;
            while (lo < hi) {   // last frame whose tile_begin <= t
                const int mid = (lo + hi + 1) >> 1;
                if (p.frames[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
            }
            const FrameDesc f = p.frames[lo];
            const int local = (int)(t - f.tile_begin);
            TileCtx tc;
            tc.img = f.img; tc.dtype = f.dtype; tc.H = f.h; tc.W = f.w; tc.pitch = f.pitch; tc.frame = lo;
            tc.x0 = (local % f.n_strips) * TX;
            const int band = local / f.n_strips;
            const int bh = (f.n_bands == 1) ? f.h : p.band;
            tc.y0 = band * bh;
            tc.y1 = min(f.h, tc.y0 + bh);
            tc.blobs = p.blobs + f.blob_off;
            tc.count = p.count + lo;
            process_tile(p, sm, ss, tc);
        }
        if (tid == 0) {
            __threadfence();
            const int d = atomicAdd(p.done_counter, 1);
            if (d == (int)gridDim.x - 1) {
                atomicExch(p.tile_counter, 0);
                atomicExch(p.done_counter, 0);
            }
        }
    }

    if (p.mode == MODE_SOFT || p.mode == MODE_BWD) {
        __syncthreads();
        if (p.mode == MODE_SOFT) {
            for (int q = tid; q < p.nbins; q += NTHREADS)
                if (ss.soft[q] != 0.0f) atomicAdd(&p.soft_out[q], ss.soft[q]);
        } else {
            for (int q = tid; q < p.P; q += NTHREADS) {
                if (ss.dc[q] != 0.0f) atomicAdd(&p.dc_acc[q], (double)ss.dc[q]);
                if (ss.dt[q] != 0.0f) atomicAdd(&p.dt_acc[q], (double)ss.dt[q]);
            }
        }
    }
}

cudaError_t launch_fused(const FusedParams& p, int grid, cudaStream_t s) {
    const bool batched = p.frames != nullptr;
    cudaError_t e;
    if (batched) {
        e = cudaFuncSetAttribute(dog_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 p.smem_bytes);
        if (e != cudaSuccess) return e;
        dog_fused_kernel<true><<<grid, NTHREADS, p.smem_bytes, s>>>(p);
    } else {
        e = cudaFuncSetAttribute(dog_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 p.smem_bytes);
        if (e != cudaSuccess) return e;
        dog_fused_kernel<false><<<grid, NTHREADS, p.smem_bytes, s>>>(p);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Resolve: one warp per queued strip-edge candidate.  The D values of the
// neighbouring strip's edge column are recomputed with the fused kernel's
// exact operation order (horizontal then vertical FMA chains from zero in
// ascending tap order, then c * (a - b)), so they equal what that strip held.
__device__ float level_value(const ResolveParams& p, const void* img, int dtype, int H, int W,
                             int pitch, int m, int y, int x, float* hbuf, int lane) {
    const int r = p.r[m];
    const float* w = p.w + p.woff[m];
    // horizontal chains of rows y-r .. y+r at column x
    for (int t = lane; t <= 2 * r; t += 32) {
        const int yy = refl(y - r + t, H);
        float acc = 0.0f;
        for (int s = 0; s <= 2 * r; ++s) {
            const int j = s >= r ? s - r : r - s;
            acc = __fmaf_rn(__ldg(w + j), load_px(img, dtype, pitch, yy, refl(x - r + s, W)), acc);
        }
        hbuf[t] = acc;
    }
    __syncwarp();
    float acc = 0.0f;
    for (int t = 0; t <= 2 * r; ++t) {
        const int j = t >= r ? t - r : r - t;
        acc = __fmaf_rn(__ldg(w + j), hbuf[t], acc);
    }
    __syncwarp();
    return acc;
}

__global__ void __launch_bounds__(128) dog_resolve_kernel(const __grid_constant__ ResolveParams p) {
    __shared__ float hbuf_all[4][2 * DOG_MAX_RADIUS + 1];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* hbuf = hbuf_all[warp];
    const int npend = min(*p.pend_count, p.pend_cap);
    for (int q = blockIdx.x * 4 + warp; q < npend; q += gridDim.x * 4) {
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
        const int lx = e.x % TX;
        const int xn = (lx == 0) ? e.x - 1 : e.x + 1;   // the column held by the other strip
        bool keep = true;
        const int l = e.level;
        // L at levels l-1 .. l+2 (those in range) and rows y-1 .. y+1
        float Lv[4][3];
        for (int mi = 0; mi < 4; ++mi) {
            const int m = l - 1 + mi;
            for (int yi = 0; yi < 3; ++yi) {
                const int y = e.y - 1 + yi;
                Lv[mi][yi] = 0.0f;
                if (m < 0 || m >= p.K || y < 0 || y >= H) continue;
                Lv[mi][yi] = level_value(p, img, dtype, H, W, pitch, m, y, xn, hbuf, lane);
            }
        }
        for (int mi = 0; mi < 3; ++mi) {
            const int ll = l - 1 + mi;
            if (ll < 0 || ll >= p.P) continue;
            for (int yi = 0; yi < 3; ++yi) {
                const int y = e.y - 1 + yi;
                if (y < 0 || y >= H) continue;
                const float d = __fmul_rn(__ldg(p.c + ll), __fsub_rn(Lv[mi][yi], Lv[mi + 1][yi]));
                if (d > e.response) keep = false;
            }
        }
        if (lane == 0 && keep) {
            if (p.mode == MODE_CANDIDATES) {
                const int idx = atomicAdd(count, 1);
                if (idx < p.cap) {
                    dog_blob bl;
                    bl.x = e.x; bl.y = e.y; bl.level = l; bl.sigma = __ldg(p.c + p.P + l); bl.response = e.response;
                    blobs[idx] = bl;
                } else {
                    atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                }
            } else {
                const float s = 1.0f / (1.0f + __expf(-(e.response - p.thr) * p.inv_T));
                if (p.mode == MODE_SOFT) {
                    for (int b = 0; b < p.nbins; ++b) {
                        const float k = p.kappa[l * p.nbins + b];
                        if (k != 0.0f) atomicAdd(&p.soft_out[b], s * k);
                    }
                } else {
                    float gk = 0.0f, gdk = 0.0f;
                    for (int b = 0; b < p.nbins; ++b) {
                        gk += p.gH[b] * p.kappa[l * p.nbins + b];
                        gdk += p.gH[b] * p.dkappa[l * p.nbins + b];
                    }
                    const float cl = __ldg(p.c + l);
                    const float G = gk * s * (1.0f - s) * p.inv_T;
                    atomicAdd(&p.A[((size_t)l * H + e.y) * W + e.x], cl * G);
                    atomicAdd(&p.A[((size_t)(l + 1) * H + e.y) * W + e.x], -cl * G);
                    atomicAdd(&p.dc_acc[l], (double)(G * e.response / cl));
                    atomicAdd(&p.dt_acc[l], (double)(s * gdk));
                }
            }
        }
        __syncwarp();
    }
}

cudaError_t launch_resolve(const ResolveParams& p, int max_pending, cudaStream_t s) {
    int grid = (max_pending + 3) / 4;
    if (grid < 1) grid = 1;
    if (grid > 152 * 16) grid = 152 * 16;
    dog_resolve_kernel<<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched set-up: per-frame descriptors and the exclusive prefix sum of tiles
// (strips x row bands) that the persistent kernel walks.  One CTA.
__global__ void __launch_bounds__(1024) dog_batch_prep_kernel(const dog_frame* frames, int n, int band,
                                                              int blob_cap, FrameDesc* desc,
                                                              long long* cand_off, long long* out_off,
                                                              int* hw, long long* ntiles) {
    __shared__ long long carry;
    __shared__ long long wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
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
            d.dtype = fr.dtype;
            d.blob_off = (long long)f * blob_cap;
            d.n_strips = (fr.w + TX - 1) / TX;
            d.n_bands = (band > 0 && band < fr.h) ? (fr.h + band - 1) / band : 1;
            tiles = (long long)d.n_strips * d.n_bands;
            cand_off[f] = (long long)f * blob_cap;
            out_off[f] = fr.blob_off;
            hw[2 * f] = fr.h;
            hw[2 * f + 1] = fr.w;
        }
        // block-wide inclusive scan of tiles
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        long long x = tiles;
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
        if (f < n) {
            d.tile_begin = carry + incl - tiles;
            desc[f] = d;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ntiles = carry;
}

cudaError_t launch_batch_prep(const dog_frame* frames, int n, int band, int blob_cap, FrameDesc* desc,
                              long long* cand_off, long long* out_off, int* hw, long long* ntiles,
                              cudaStream_t s) {
    dog_batch_prep_kernel<<<1, 1024, 0, s>>>(frames, n, band, blob_cap, desc, cand_off, out_off, hw, ntiles);
    return cudaGetLastError();
}

}  // namespace dogk
