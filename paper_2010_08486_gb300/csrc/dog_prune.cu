// Overlap pruning (Sec. 4.1) and blob-volume histogram (Sec. 4) on sm_103a.
//
// Pruning.  The paper coalesces blobs whose normalised overlap exceeds a
// threshold.  Read as a greedy pass in priority order (response descending,
// then level, y, x), a candidate is accepted iff no accepted candidate of
// higher priority conflicts with it; a rejected candidate joins the
// highest-priority accepted candidate it conflicts with.  That outcome is the
// lexicographically-first maximal independent set of the conflict graph in
// priority order, which this kernel computes in parallel rounds: a candidate
// becomes IN once every higher-priority neighbour is OUT, and OUT once any is
// IN.  Round count is bounded by the candidate count (each round settles at
// least the highest-priority undecided candidate).
//
// Conflict test.  Centres are integer pixels, so the squared distance d2 is an
// integer; for a pair of planes (a, b) the host precomputes the smallest
// integer d2 at which the double-precision overlap drops to the threshold
// (overlap decreases with distance).  Two candidates conflict iff
// d2 < d2thr[a][b] -- the device evaluates no transcendental function.
// Neighbours are found through a hashed grid with cells of edge >= the
// largest conflict distance, so all conflicts lie in the 3x3 adjacent cells.
#include <cuda_runtime.h>

#include <atomic>

#include "dog_internal.cuh"

namespace dogk {

// Histogram bin of one blob (Sec. 4): a blob whose stored sigma equals its
// plane's single-precision sigma takes its plane's precomputed bin; another
// sigma (a coalesced mean) is binned by log volume (LOGV) or by the nearest
// ladder radius in log space (LADDER).
__device__ __forceinline__ int hist_bin(const dog_blob& b, const HistParams& p) {
    const int l = min(max(b.level, 0), p.P - 1);
    if (b.sigma == p.sig_f[l]) return p.level_bin[l];
    if (p.mode == DOG_HIST_LADDER) {
        const double ls = log((double)b.sigma);
        int best = 0;
        double bd = fabs(ls - p.log_sig[0]);
        for (int q = 1; q < p.P; ++q) {
            const double d = fabs(ls - p.log_sig[q]);
            if (d < bd) { bd = d; best = q; }
        }
        return best;
    }
    const double span = p.log_hi - p.log_lo;
    const double t = (p.P >= 2 && span > 0.0) ? (log((double)b.sigma) - p.log_lo) / span : 0.0;
    double fb = floor((double)p.nbins * t);
    fb = fmin(fmax(fb, 0.0), (double)(p.nbins - 1));
    return (int)fb;
}

__device__ __forceinline__ double blob_volume(float sigma) {
    const double r = 1.4142135623730951 * (double)sigma;
    return 4.0 / 3.0 * 3.141592653589793 * r * r * r;
}


constexpr int PRUNE_THREADS = 1024;
constexpr int NBUCKET = 4096;
enum { ST_UND = 0, ST_IN = 1, ST_OUT = 2 };

__device__ __forceinline__ bool higher(const dog_blob& a, const dog_blob& b) {
    if (a.response != b.response) return a.response > b.response;
    if (a.level != b.level) return a.level < b.level;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
}

__device__ __forceinline__ int plane_of(const dog_blob& b, int P) { return min(max(b.level, 0), P - 1); }

__device__ __forceinline__ unsigned bucket_of(int cx, int cy) {
    return (((unsigned)cx * 73856093u) ^ ((unsigned)cy * 19349663u)) & (NBUCKET - 1);
}

struct PruneSmem {
    int bcount[NBUCKET];
    int boff[NBUCKET + 1];
    int d2[MAX_LEVELS * MAX_LEVELS];
    int changed;
    int scan_carry;
};

// The buckets of the 3x3 cells around (cx, cy).  Two cells may hash to the
// same bucket; every use below is unaffected by visiting a candidate twice
// (an any-of test, a maximum, a search for the next member in priority order).
__device__ __forceinline__ int neighbour_buckets(int cx, int cy, unsigned* bk) {
    int nb = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) bk[nb++] = bucket_of(cx + dx, cy + dy);
    return nb;
}

// Volume histogram of one frame's pruned blobs (out[0 .. out_count[f])),
// written whole by the frame's CTA (no other CTA touches it).
__device__ void frame_hist(const PruneParams& p, PruneSmem& s, const dog_blob* out, int f) {
    const HistParams& hp = p.hist;
    const int tid = threadIdx.x;
    const int nbo = (hp.mode == DOG_HIST_LADDER) ? hp.P : hp.nbins;
    unsigned* hc = reinterpret_cast<unsigned*>(s.bcount);
    double* hv = reinterpret_cast<double*>(s.boff);
    __syncthreads();
    for (int q = tid; q < nbo; q += PRUNE_THREADS) { hc[q] = 0u; hv[q] = 0.0; }
    __syncthreads();
    const int nout = min(p.out_count[f], p.cap_out);
    for (int i = tid; i < nout; i += PRUNE_THREADS) {
        const dog_blob b = out[i];
        const int bin = hist_bin(b, hp);
        atomicAdd(&hc[bin], 1u);
        if (hp.vol) atomicAdd(&hv[bin], blob_volume(b.sigma));
    }
    __syncthreads();
    for (int q = tid; q < nbo; q += PRUNE_THREADS) {
        hp.hist[(size_t)f * nbo + q] = hc[q];
        if (hp.vol) hp.vol[(size_t)f * nbo + q] = hv[q];
    }
}

// Frames with at most PRUNE_SMEM_CAND candidates run every pass on
// shared-memory copies of the candidates and the per-candidate arrays
// (dynamic shared memory, PRUNE_DYN_BYTES); larger ones work in global memory.
constexpr int PRUNE_SMEM_CAND = 4096;
constexpr int PRUNE_DYN_BYTES = PRUNE_SMEM_CAND * ((int)sizeof(dog_blob) + 3 * (int)sizeof(int));

__global__ void __launch_bounds__(PRUNE_THREADS) dog_prune_kernel(const __grid_constant__ PruneParams p) {
    __shared__ PruneSmem s;
    extern __shared__ int4 prune_dyn[];
    const int f = blockIdx.x;
    const int tid = threadIdx.x;
    const long long coff = p.cand_off ? p.cand_off[f] : 0;
    const long long ooff = p.out_off ? p.out_off[f] : 0;
    const dog_blob* cand = p.cand + coff;
    int* state = p.state + coff;
    int* target = p.target + coff;
    int* order = p.order + coff;
    dog_blob* out = p.out + ooff;
    const int n = min(p.cand_count[f], p.cap_in);
    if (n <= PRUNE_SMEM_CAND && p.mode != DOG_PRUNE_OFF) {
        dog_blob* sc = reinterpret_cast<dog_blob*>(prune_dyn);
        int* si = reinterpret_cast<int*>(sc + PRUNE_SMEM_CAND);
        for (int i = tid; i < n; i += PRUNE_THREADS) sc[i] = cand[i];
        cand = sc;
        state = si;
        target = si + PRUNE_SMEM_CAND;
        order = si + 2 * PRUNE_SMEM_CAND;
        // made visible by the first __syncthreads below
    }

    if (p.mode == DOG_PRUNE_OFF) {
        for (int i = tid; i < n; i += PRUNE_THREADS) {
            if (i < p.cap_out) out[i] = cand[i];
        }
        if (tid == 0) {
            p.out_count[f] = n;
            if (n > p.cap_out) atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
        }
        if (p.hist.hist) frame_hist(p, s, out, f);
        return;
    }

    for (int q = tid; q < NBUCKET; q += PRUNE_THREADS) s.bcount[q] = 0;
    for (int q = tid; q < p.P * p.P; q += PRUNE_THREADS) s.d2[q] = p.d2thr[q];
    if (tid == 0) { s.scan_carry = 0; p.out_count[f] = 0; }
    __syncthreads();
    const int cell = p.cell;

    // 1. counting sort of candidate indices by hashed cell
    for (int i = tid; i < n; i += PRUNE_THREADS) {
        const dog_blob b = cand[i];
        const unsigned bk = bucket_of(b.x / cell, b.y / cell);
        target[i] = (int)bk;
        atomicAdd(&s.bcount[bk], 1);
        state[i] = ST_UND;
    }
    __syncthreads();
    // exclusive scan of the bucket counts (4 per thread, sequential carry across chunks)
    for (int base = 0; base < NBUCKET; base += PRUNE_THREADS) {
        const int v = s.bcount[base + tid];
        int x = v;
        // warp inclusive scan
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ int wsum[32];
        if (lane == 31) wsum[warp] = x;
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
        const int incl = x + (warp > 0 ? wsum[warp - 1] : 0);
        s.boff[base + tid] = s.scan_carry + incl - v;
        __syncthreads();
        if (tid == PRUNE_THREADS - 1) s.scan_carry += incl;
        __syncthreads();
    }
    if (tid == 0) s.boff[NBUCKET] = s.scan_carry;
    for (int q = tid; q < NBUCKET; q += PRUNE_THREADS) s.bcount[q] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += PRUNE_THREADS) {
        const int bk = target[i];
        const int pos = s.boff[bk] + atomicAdd(&s.bcount[bk], 1);
        order[pos] = i;
    }
    __syncthreads();

    // 2. rounds of the independent-set rule
    volatile int* vstate = state;
    for (int round = 0; round <= n + 1; ++round) {
        if (tid == 0) s.changed = 0;
        __syncthreads();
        for (int i = tid; i < n; i += PRUNE_THREADS) {
            if (vstate[i] != ST_UND) continue;
            const dog_blob bi = cand[i];
            unsigned bk[9];
            neighbour_buckets(bi.x / cell, bi.y / cell, bk);
            bool any_in = false, any_und = false;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (any_in) break;
                for (int k = s.boff[bk[q]]; k < s.boff[bk[q] + 1]; ++k) {
                    const int j = order[k];
                    if (j == i) continue;
                    const dog_blob bj = cand[j];
                    const int dx = bj.x - bi.x, dy = bj.y - bi.y;
                    if (dx * dx + dy * dy >= s.d2[plane_of(bi, p.P) * p.P + plane_of(bj, p.P)]) continue;
                    if (!higher(bj, bi)) continue;
                    const int st = vstate[j];
                    if (st == ST_IN) { any_in = true; break; }
                    if (st == ST_UND) any_und = true;
                }
            }
            if (any_in) { vstate[i] = ST_OUT; s.changed = 1; }
            else if (!any_und) { vstate[i] = ST_IN; s.changed = 1; }
        }
        __syncthreads();
        if (!s.changed) break;
        __syncthreads();
    }

    // 3. every rejected candidate joins its highest-priority accepted neighbour
    for (int i = tid; i < n; i += PRUNE_THREADS) {
        target[i] = -1;
        if (state[i] != ST_OUT) continue;
        const dog_blob bi = cand[i];
        unsigned bk[9];
        neighbour_buckets(bi.x / cell, bi.y / cell, bk);
        int best = -1;
#pragma unroll
        for (int q = 0; q < 9; ++q)
            for (int k = s.boff[bk[q]]; k < s.boff[bk[q] + 1]; ++k) {
                const int j = order[k];
                if (j == i || (state[j] & 3) != ST_IN) continue;
                const dog_blob bj = cand[j];
                const int dx = bj.x - bi.x, dy = bj.y - bi.y;
                if (dx * dx + dy * dy >= s.d2[plane_of(bi, p.P) * p.P + plane_of(bj, p.P)]) continue;
                if (!higher(bj, bi)) continue;
                if (best < 0 || higher(bj, cand[best])) best = j;
            }
        target[i] = best;
        if (best < 0) atomicCAS(p.status, 0, (int)DOG_ERR_INVALID);   // cannot happen
        else atomicAdd(&state[best], 4);   // member count of an accepted candidate, above the state bits
    }
    __syncthreads();

    // 4. accepted blobs: group mean sigma summed in visiting order, then compaction
    for (int a = tid; a < n; a += PRUNE_THREADS) {
        if ((state[a] & 3) != ST_IN) continue;
        const int nmem = state[a] >> 2;
        const dog_blob ba = cand[a];
        double sum = p.sig[plane_of(ba, p.P)];
        int cnt = 1;
        bool mixed = false;
        if (p.mode == DOG_PRUNE_COALESCE && nmem > 0) {
            unsigned bk[9];
            neighbour_buckets(ba.x / cell, ba.y / cell, bk);
            int prev = a;
            for (;;) {
                // next member after `prev` in priority order
                int nxt = -1;
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    for (int k = s.boff[bk[q]]; k < s.boff[bk[q] + 1]; ++k) {
                        const int j = order[k];
                        if (target[j] != a) continue;
                        const dog_blob bj = cand[j];
                        if (!higher(cand[prev], bj)) continue;
                        if (nxt < 0 || higher(bj, cand[nxt])) nxt = j;
                    }
                if (nxt < 0) break;
                const dog_blob bn = cand[nxt];
                sum += p.sig[plane_of(bn, p.P)];
                ++cnt;
                mixed |= (bn.level != ba.level);
                prev = nxt;
                if (cnt > nmem) break;   // all members visited
            }
        }
        dog_blob o = ba;
        o.sigma = mixed ? (float)(sum / (double)cnt) : (float)p.sig[plane_of(ba, p.P)];
        const int idx = atomicAdd(&p.out_count[f], 1);
        if (idx < p.cap_out) out[idx] = o;
        else atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
    }
    // 5. optional: this frame's volume histogram
    if (p.hist.hist) frame_hist(p, s, out, f);
}

// Set once per device (not on every launch, so launches can be graph-captured);
// atomic because the launcher may be called from several host threads.
static std::atomic<bool> g_prune_attr[64];

cudaError_t launch_prune(const PruneParams& p, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!g_prune_attr[dev & 63].load(std::memory_order_acquire)) {
        // setting the attribute twice from two threads is harmless
        e = cudaFuncSetAttribute(dog_prune_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PRUNE_DYN_BYTES);
        if (e != cudaSuccess) return e;
        g_prune_attr[dev & 63].store(true, std::memory_order_release);
    }
    dog_prune_kernel<<<p.n_frames, PRUNE_THREADS, PRUNE_DYN_BYTES, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Histogram: one CTA row per frame, shared-memory bins, one global atomic per
// non-empty bin and CTA.
__global__ void __launch_bounds__(256) dog_hist_kernel(const __grid_constant__ HistParams p) {
    __shared__ unsigned hc[DOG_MAX_NBINS];
    __shared__ double hv[DOG_MAX_NBINS];
    const int f = blockIdx.y;
    const int nbo = (p.mode == DOG_HIST_LADDER) ? p.P : p.nbins;
    for (int q = threadIdx.x; q < nbo; q += blockDim.x) { hc[q] = 0u; hv[q] = 0.0; }
    __syncthreads();
    const long long off = p.off ? p.off[f] : 0;
    const int n = min(p.count[f], p.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const dog_blob b = p.blobs[off + i];
        const int bin = hist_bin(b, p);
        atomicAdd(&hc[bin], 1u);
        if (p.vol) atomicAdd(&hv[bin], blob_volume(b.sigma));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nbo; q += blockDim.x) {
        if (hc[q]) atomicAdd(&p.hist[(size_t)f * nbo + q], hc[q]);
        if (p.vol && hv[q] != 0.0) atomicAdd(&p.vol[(size_t)f * nbo + q], hv[q]);
    }
}

cudaError_t launch_hist(const HistParams& p, cudaStream_t s) {
    dim3 grid(4, p.n_frames);
    dog_hist_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void dog_ring_push_kernel(const uint32_t* hist, int nbins, uint32_t* ring, int window,
                                     uint32_t* sum, int32_t* head) {
    const int h = *head;
    const int slot = ((h % window) + window) % window;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const uint32_t old = (h >= window) ? ring[(size_t)slot * nbins + b] : 0u;
        const uint32_t nw = hist[b];
        ring[(size_t)slot * nbins + b] = nw;
        sum[b] = sum[b] - old + nw;
    }
    __syncthreads();
    if (threadIdx.x == 0) *head = h + 1;
}

cudaError_t launch_ring_push(const uint32_t* hist, int nbins, uint32_t* ring, int window, uint32_t* sum,
                             int32_t* head, cudaStream_t s) {
    dog_ring_push_kernel<<<1, 256, 0, s>>>(hist, nbins, ring, window, sum, head);
    return cudaGetLastError();
}

// One CTA per stream walks the batch in order and pushes that stream's frames.
__global__ void dog_ring_push_batched_kernel(const uint32_t* hists, const int32_t* ids, int n, int nbins,
                                             uint32_t* rings, int window, uint32_t* sums, int32_t* heads) {
    const int sid = blockIdx.x;
    uint32_t* ring = rings + (size_t)sid * window * nbins;
    uint32_t* sum = sums + (size_t)sid * nbins;
    int h = heads[sid];
    for (int f = 0; f < n; ++f) {
        if (ids[f] != sid) continue;
        const int slot = h % window;
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
            const uint32_t old = (h >= window) ? ring[(size_t)slot * nbins + b] : 0u;
            const uint32_t nw = hists[(size_t)f * nbins + b];
            ring[(size_t)slot * nbins + b] = nw;
            sum[b] = sum[b] - old + nw;
        }
        ++h;
        __syncthreads();
    }
    if (threadIdx.x == 0) heads[sid] = h;
}

cudaError_t launch_ring_push_batched(const uint32_t* hists, const int32_t* ids, int n, int nbins, int n_streams,
                                     uint32_t* rings, int window, uint32_t* sums, int32_t* heads, cudaStream_t s) {
    dog_ring_push_batched_kernel<<<n_streams, 128, 0, s>>>(hists, ids, n, nbins, rings, window, sums, heads);
    return cudaGetLastError();
}

}  // namespace dogk
