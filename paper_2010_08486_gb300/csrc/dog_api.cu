// C ABI of the sm_103a DoG detector: handle set-up on the host and the
// stream-ordered entry points declared in include/dog.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "dog_internal.cuh"

namespace dogk {
cudaError_t launch_ring_push(const uint32_t* hist, int nbins, uint32_t* ring, int window, uint32_t* sum,
                             int32_t* head, cudaStream_t s);
cudaError_t launch_ring_push_batched(const uint32_t* hists, const int32_t* ids, int n, int nbins, int n_streams,
                                     uint32_t* rings, int window, uint32_t* sums, int32_t* heads, cudaStream_t s);
// differentiable form (dog_soft.cu)
int soft_forward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig, float* out,
                 dog_soft_max* rec, int rec_cap, int* rec_count, cudaStream_t s);
int soft_backward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig,
                  const float* gH, float* gimg, float* gsig, cudaStream_t s);
int soft_backward_rec(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig,
                      const dog_soft_max* rec, const int* rec_count, int rec_cap, const float* gH, float* gimg,
                      float* gsig, cudaStream_t s);
}  // namespace dogk

using namespace dogk;

// ---------------------------------------------------------------------------
#define DOG_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            return e_ == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA; \
        }                                                     \
    } while (0)

struct dog_handle {
    dog_config cfg;
    std::vector<double> explicit_sig;
    int K = 0, P = 0, R = 0;
    int geom = 0;
    std::vector<double> sig;
    std::vector<int> rad;
    std::vector<double> norm;
    std::vector<int> woff;
    std::vector<int> hoff;   // the horizontal pass's copy of the taps
    int w_total = 0;
    int num_sms = 0;
    int band = 0;          // 0: whole frame
    int ctas_per_sm = 1;
    FusedParams base{};
    // device tables
    float* d_w = nullptr;
    float* d_c = nullptr;          // P normalisation coefficients, then P plane sigmas (float)
    double* d_sig64 = nullptr;     // P plane sigmas (double)
    int* d_d2thr = nullptr;
    int cell = 1;
    float* d_sigf = nullptr;
    int* d_levbin = nullptr;
    double* d_logsig = nullptr;
    double log_lo = 0.0, log_hi = 0.0;
    // workspace
    dog_blob* d_cand = nullptr;
    int cand_cap = 0;
    int* d_counts = nullptr;       // [0] candidates [1] pending [2] tile counter [3] done counter
    Pending* d_pend = nullptr;
    int pend_cap = 0;
    int* d_state = nullptr;
    int* d_target = nullptr;
    int* d_order = nullptr;
    int* d_status = nullptr;
    // batched workspace (grown on demand)
    int batch_cap = 0;
    FrameDesc* d_desc = nullptr;
    long long* d_cand_off = nullptr;
    long long* d_out_off = nullptr;
    int* d_hw = nullptr;
    long long* d_ntiles = nullptr;
    dog_blob* d_bcand = nullptr;
    int* d_bstate = nullptr;
    int* d_btarget = nullptr;
    int* d_border = nullptr;
    int* d_bcounts = nullptr;
    Pending* d_bpend = nullptr;
    int bpend_cap = 0;
    // contrast stretch: histogram and limits of a single frame, and of each
    // frame of a batch (grown with the batch workspace)
    int* d_shist = nullptr;
    int* d_slohi = nullptr;
    int* d_bshist = nullptr;
    int* d_bslohi = nullptr;
    // FFT backend (created by its first call)
    FftWS* fft = nullptr;
    bool direct_ok = true;   // the fused kernel's shared memory fits this device
    // differentiable form
    void* soft_ws = nullptr;
    cudaStream_t last = nullptr;
    // measurement of the fused kernel
    bool prof = false;
    std::vector<cudaEvent_t> ev;   // start/stop pairs
    int ev_used = 0;
};

namespace dogk {
// accessors used by dog_soft.cu (keeps dog_handle private to this file)
const FusedParams& handle_base(const dog_handle* h) { return h->base; }
int handle_K(const dog_handle* h) { return h->K; }
int handle_P(const dog_handle* h) { return h->P; }
const std::vector<int>& handle_radii(const dog_handle* h) { return h->rad; }
const std::vector<double>& handle_sigmas(const dog_handle* h) { return h->sig; }
const dog_config& handle_cfg(const dog_handle* h) { return h->cfg; }
int handle_band(const dog_handle* h) { return h->band; }
int* handle_status(dog_handle* h) { return h->d_status; }
void*& handle_soft_ws(dog_handle* h) { return h->soft_ws; }
void handle_set_last(dog_handle* h, cudaStream_t s) { h->last = s; }

constexpr int PROF_MAX = 65536;

// Launch the fused kernel, bracketed by profiling events when enabled.
cudaError_t timed_fused(dog_handle* h, const FusedParams& p, int grid, cudaStream_t s) {
    const bool timed = h->prof && h->ev_used < PROF_MAX;
    if (timed) {
        while ((int)h->ev.size() < 2 * (h->ev_used + 1)) {
            cudaEvent_t e;
            cudaError_t x = cudaEventCreate(&e);
            if (x != cudaSuccess) return x;
            h->ev.push_back(e);
        }
        cudaError_t x = cudaEventRecord(h->ev[2 * h->ev_used], s);
        if (x != cudaSuccess) return x;
    }
    cudaError_t e = launch_fused(p, grid, s);
    if (e != cudaSuccess) return e;
    if (timed) {
        e = cudaEventRecord(h->ev[2 * h->ev_used + 1], s);
        h->ev_used++;
    }
    return e;
}
}  // namespace dogk

// ---------------------------------------------------------------------------
// host arithmetic

static double disc_overlap(double d, double ra, double rb) {
    // area of the intersection of two discs at distance d, over the smaller disc's area,
    // as the sum of the two circular segments cut by the common chord
    const double rmin = std::min(ra, rb);
    if (d >= ra + rb) return 0.0;
    if (d <= std::fabs(ra - rb)) return 1.0;
    const double xa = (d * d + ra * ra - rb * rb) / (2.0 * d);  // centre a to chord
    const double xb = d - xa;                                   // centre b to chord
    auto segment = [](double r, double x) {
        double c = x / r;
        c = std::min(1.0, std::max(-1.0, c));
        const double h2 = std::max(0.0, r * r - x * x);
        return r * r * std::acos(c) - x * std::sqrt(h2);
    };
    const double area = segment(ra, xa) + segment(rb, xb);
    return area / (M_PI * rmin * rmin);
}

namespace dogk {
int conflict_d2(double sa, double sb, double thr);
}

int dogk::conflict_d2(double sa, double sb, double thr) {
    const double ra = std::sqrt(2.0) * sa, rb = std::sqrt(2.0) * sb;
    long long lo = 0, hi = (long long)std::ceil((ra + rb) * (ra + rb)) + 1;
    // smallest integer d2 with overlap(sqrt(d2)) <= thr; overlap is non-increasing in d2
    if (disc_overlap(0.0, ra, rb) <= thr) return 0;
    while (lo + 1 < hi) {
        const long long mid = (lo + hi) / 2;
        if (disc_overlap(std::sqrt((double)mid), ra, rb) <= thr) hi = mid; else lo = mid;
    }
    return (int)hi;
}

static int ceil_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

static int status_from(cudaError_t e) {
    if (e == cudaSuccess) return DOG_OK;
    return e == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA;
}

// Allocation failures injected by dog_test_fail_alloc: the number of
// workspace allocations still allowed before one fails (-1: none fails).
static std::atomic<int> g_fail_after{-1};

template <class T>
static cudaError_t dalloc(T** p, size_t n) {
    int k = g_fail_after.load();
    while (k >= 0 && !g_fail_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) {   // this allocation is the injected failure; later ones succeed again
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(n, 1));
}

static void free_all(dog_handle* h) {
    void* ptrs[] = {h->d_w, h->d_c, h->d_sig64, h->d_d2thr, h->d_sigf, h->d_levbin, h->d_logsig,
                    h->d_cand, h->d_counts, h->d_pend, h->d_state, h->d_target, h->d_order,
                    h->d_status, h->d_desc, h->d_cand_off, h->d_out_off, h->d_hw, h->d_ntiles,
                    h->d_bcand, h->d_bstate, h->d_btarget, h->d_border, h->d_bcounts, h->d_bpend,
                    h->d_shist, h->d_slohi, h->d_bshist, h->d_bslohi};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

namespace dogk { void soft_free(dog_handle* h); }

// Balance levels over the nw producer warps of a kernel form (every block,
// all of them wait for the slowest at a barrier).  Per level the cost is two
// passes of tpad/8 tap blocks plus a fixed cost (set-up, pipeline fill and
// drain of both passes) of about 1.7 tap blocks of both passes (clock64 phase
// timers).  Over 12 warps: first-fit decreasing at the smallest capacity that
// packs all levels (raised one unit at a time from the larger of the average
// load and the largest level); on the 25-level ladder this gives a largest
// load of 124 units where longest-processing-time-first gives 134, 2% faster
// measured.  Over 8 warps: longest processing time first (each level, largest
// first, to the least loaded warp), which spreads the levels over all warps
// and measured up to 5% faster there than first-fit decreasing.
// A level whose 2r + 1 taps are one past a multiple of 8 runs its last tap
// alone (8 FMAs instead of a block of 64, no further loads): 8 units less.
static long long level_cost(const LevelInfo& L) {
    const bool tail = ((2 * L.r + 1) & 7) == 1;
    return 10 * (L.tpad / 8) + 17 - (tail ? 8 : 0);
}

static void assign_levels(dog_handle* h, int nw) {
    const int K = h->K;
    std::vector<long long> cost(K);
    long long total = 0, biggest = 0;
    for (int i = 0; i < K; ++i) {
        cost[i] = level_cost(h->base.lv[i]);
        total += cost[i];
        biggest = std::max(biggest, cost[i]);
    }
    std::vector<int> idx(K), owner(K);
    for (int i = 0; i < K; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    if (nw == 8) {
        long long load[NWARPS] = {0};
        for (int i : idx) {
            int best = 0;
            for (int w = 1; w < nw; ++w)
                if (load[w] < load[best]) best = w;
            load[best] += cost[i];
            owner[i] = best;
        }
    } else {
        for (long long cap = std::max(biggest, (total + nw - 1) / nw);; ++cap) {
            long long load[NWARPS] = {0};
            bool fits = true;
            for (int i : idx) {
                int w = 0;
                while (w < nw && load[w] + cost[i] > cap) ++w;
                if (w == nw) { fits = false; break; }
                load[w] += cost[i];
                owner[i] = w;
            }
            if (fits) break;   // ends at the latest when cap reaches the total
        }
    }
    h->base.nw = nw;
    for (int w = 0; w < NWARPS; ++w) h->base.warp_nlev[w] = 0;
    for (int i : idx) h->base.warp_lev[owner[i]][h->base.warp_nlev[owner[i]]++] = (unsigned char)i;
}

// Kernel form for a ladder when none is set: 12 producer warps for long
// ladders whose largest level fits an even share of 12 warps (there the
// extra warps hide latency), else 8 with more registers each (a few large
// levels: their warps set the pace).  Measured on 96 frames of 1024 x 1024
// (ms per launch, 12 / 8 warps): 25 levels sigma 0.8..7.9 (largest level 107
// units of 1395) 10.82 / 11.72; 14 levels sigma 2..12.3 (147 of 1148)
// 12.59 / 10.98; 12 levels sigma 1..11.6 (137 of 824) 9.95 / 9.33; 24 levels
// sigma 2..2.8 (47 of 1128) 12.27 / 11.39, which this rule gets wrong (the
// autotuner times both forms).
static int default_producer_warps(const dog_handle* h) {
    long long total = 0, biggest = 0;
    for (int i = 0; i < h->K; ++i) {
        const long long c = level_cost(h->base.lv[i]);
        total += c;
        biggest = std::max(biggest, c);
    }
    return (h->K >= 20 && 12 * biggest <= total) ? 12 : 8;
}

extern "C" {

int dog_config_default(dog_config* c) {
    if (!c) return DOG_ERR_INVALID;
    std::memset(c, 0, sizeof(*c));
    c->n_levels = 0;
    c->sigmas = nullptr;
    c->min_sigma = 1.0;
    c->max_sigma = 10.0;
    c->ratio = 1.6;
    c->ladder = DOG_LADDER_GEOM;
    c->truncate = 4.0;
    c->threshold = 0.1;
    c->overlap = 0.5;
    c->norm = DOG_NORM_DERIV;
    c->prune = DOG_PRUNE_COALESCE;
    c->nbins = 32;
    c->hist_mode = DOG_HIST_LOGV;
    c->soft_T = 0.01;
    c->max_h = 1024;
    c->max_w = 1024;
    c->blob_cap = 65536;
    c->stretch_sat = 0.0;
    c->backend = DOG_BACKEND_DIRECT;
    return DOG_OK;
}

int dog_create(const dog_config* cfg, dog_t** out) {
    if (!cfg || !out) return DOG_ERR_INVALID;
    *out = nullptr;
    const dog_config& c = *cfg;
    if (!(c.truncate > 0.0) || !(c.overlap >= 0.0 && c.overlap < 1.0) || c.nbins < 1 ||
        c.nbins > DOG_MAX_NBINS || c.max_h < 1 || c.max_w < 1 || c.blob_cap < 1 ||
        !(c.soft_T > 0.0) || !(c.stretch_sat >= 0.0 && c.stretch_sat < 1.0))
        return DOG_ERR_INVALID;
    if (c.norm != DOG_NORM_DERIV && c.norm != DOG_NORM_PAPER) return DOG_ERR_INVALID;
    if (c.prune < DOG_PRUNE_COALESCE || c.prune > DOG_PRUNE_OFF) return DOG_ERR_INVALID;
    if (c.hist_mode != DOG_HIST_LOGV && c.hist_mode != DOG_HIST_LADDER) return DOG_ERR_INVALID;
    if (c.backend != DOG_BACKEND_DIRECT && c.backend != DOG_BACKEND_FFT) return DOG_ERR_INVALID;

    dog_handle* h = new (std::nothrow) dog_handle();
    if (!h) return DOG_ERR_NOMEM;
    h->cfg = c;
    // ---- ladder (Sec. 4, Eq. 1)
    std::vector<double>& sig = h->sig;
    if (c.sigmas) {
        if (c.n_levels < 3) { delete h; return DOG_ERR_INVALID; }
        sig.assign(c.sigmas, c.sigmas + c.n_levels);
        h->explicit_sig = sig;
        h->cfg.sigmas = nullptr;
    } else if (c.ladder == DOG_LADDER_ARITH) {
        if (c.n_levels < 3 || !(c.max_sigma > c.min_sigma) || !(c.min_sigma > 0.0)) { delete h; return DOG_ERR_INVALID; }
        const int n_bin = c.n_levels - 1;
        const double delta = (c.max_sigma - c.min_sigma) / (double)n_bin;
        for (int i = 0; i < c.n_levels; ++i) sig.push_back(c.min_sigma + (double)i * delta);
    } else if (c.ladder == DOG_LADDER_GEOM) {
        if (!(c.min_sigma > 0.0) || !(c.ratio > 1.0)) { delete h; return DOG_ERR_INVALID; }
        int K = c.n_levels;
        if (K <= 0) {
            if (!(c.max_sigma > c.min_sigma)) { delete h; return DOG_ERR_INVALID; }
            K = (int)std::floor(std::log(c.max_sigma / c.min_sigma) / std::log(c.ratio) + 1e-9) + 2;
        }
        for (int i = 0; i < K; ++i) sig.push_back(c.min_sigma * std::pow(c.ratio, (double)i));
        h->geom = 1;
    } else {
        delete h;
        return DOG_ERR_INVALID;
    }
    h->K = (int)sig.size();
    h->P = h->K - 1;
    if (h->K < 3) { delete h; return DOG_ERR_INVALID; }
    if (h->K > DOG_MAX_LEVELS) { delete h; return DOG_ERR_UNSUPPORTED; }
    for (int i = 0; i < h->K; ++i) {
        if (!(sig[i] > 0.0) || (i > 0 && !(sig[i] > sig[i - 1]))) { delete h; return DOG_ERR_INVALID; }
        const int r = (int)std::floor(c.truncate * sig[i] + 0.5);
        if (r < 1) { delete h; return DOG_ERR_INVALID; }
        if (r > DOG_MAX_RADIUS) { delete h; return DOG_ERR_UNSUPPORTED; }
        h->rad.push_back(r);
        h->R = std::max(h->R, r);
    }
    // ---- kernels (double, rounded to float): full taps t = 0..2r (tap t weighs
    // the sample at offset t - r), zero-padded to a multiple of 8 taps
    std::vector<float> wf;
    for (int i = 0; i < h->K; ++i) {
        const int r = h->rad[i];
        const int tpad = 8 * ((2 * r + 1 + 7) / 8);
        std::vector<double> e(2 * r + 1);
        double z = 0.0;
        for (int j = -r; j <= r; ++j) {
            e[j + r] = std::exp(-(double)j * j / (2.0 * sig[i] * sig[i]));
            z += e[j + r];
        }
        h->woff.push_back((int)wf.size());
        for (int t = 0; t < tpad; ++t) wf.push_back(t <= 2 * r ? (float)(e[t] / z) : 0.0f);
    }
    // a second copy of every level's taps for the horizontal pass: with the two
    // passes reading separate tables the fused kernel runs 35% faster than
    // with one shared table (measured; same values, same order)
    for (int i = 0; i < h->K; ++i) {
        h->hoff.push_back((int)wf.size());
        const int tpad = 8 * ((2 * h->rad[i] + 1 + 7) / 8);
        for (int t = 0; t < tpad; ++t) {
            const float v = wf[h->woff[i] + t];
            wf.push_back(v);
        }
    }
    h->w_total = (int)wf.size();
    // ---- normalisation (Eq. 3 / heat-equation finite difference)
    for (int i = 0; i < h->P; ++i)
        h->norm.push_back(c.norm == DOG_NORM_PAPER ? sig[i] : sig[i] / (sig[i + 1] - sig[i]));
    std::vector<float> cf;
    for (int i = 0; i < h->P; ++i) cf.push_back((float)h->norm[i]);
    for (int i = 0; i < h->P; ++i) cf.push_back((float)sig[i]);

    // ---- shared-memory layout of the fused kernel
    FusedParams& b = h->base;
    b.K = h->K;
    b.P = h->P;
    b.R = h->R;
    b.thr = (float)c.threshold;
    int dmin = 1 << 30, dmax = -(1 << 30);
    int off = 0;
    b.w_off = off;
    b.w_total = h->w_total;
    off += h->w_total;
    // input rows hold TX + 2R loaded columns; the padded taps of the widest
    // level read 8 further (zero) columns; an odd stride keeps the eight rows
    // read by one horizontal-pass instruction on distinct banks
    b.in_stride = (TX + 2 * h->R + 8) | 1;
    for (int i = 0; i < h->K; ++i) {
        LevelInfo& L = b.lv[i];
        L.r = h->rad[i];
        L.tpad = 8 * ((2 * L.r + 1 + 7) / 8);
        L.e = L.tpad / MB;
        L.delta = MB * L.e - L.r;
        L.ring_rows = L.tpad + MB;
        L.woff = h->woff[i];
        L.hoff = h->hoff[i];
        dmin = std::min(dmin, L.delta);
        dmax = std::max(dmax, L.delta);
    }
    b.dmin = dmin;
    b.dmax = dmax;
    // a block reads dmax - dmin + MB input rows; the next block's MB rows are
    // stored while other producer warps may still read this block's
    b.in_rows = std::max(32, ceil_pow2(dmax - dmin + 2 * MB));
    off = (off + 3) & ~3;
    b.in_off = off;
    off += b.in_rows * b.in_stride;
    off = (off + 3) & ~3;
    b.d_off = off;
    off += h->K * DSLOTS * TX;
    for (int i = 0; i < h->K; ++i) {
        off = (off + 3) & ~3;
        b.lv[i].ring_off = off;
        off += b.lv[i].ring_rows * RING_STRIDE;
    }
    b.smem_bytes = off * (int)sizeof(float);
    assign_levels(h, default_producer_warps(h));

    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete h;
        return DOG_ERR_CUDA;
    }
    // the fused kernel's shared memory must fit; an FFT-backend handle can do
    // without it (its differentiable and batched calls then report UNSUPPORTED)
    h->direct_ok = b.smem_bytes + 4096 <= optin;
    if (!h->direct_ok && c.backend == DOG_BACKEND_DIRECT) { delete h; return DOG_ERR_UNSUPPORTED; }

    // ---- pruning conflict table and histogram tables
    std::vector<int> d2(h->P * h->P);
    int maxd2 = 1;
    for (int a = 0; a < h->P; ++a)
        for (int q = 0; q < h->P; ++q) {
            d2[a * h->P + q] = conflict_d2(sig[a], sig[q], c.overlap);
            maxd2 = std::max(maxd2, d2[a * h->P + q]);
        }
    h->cell = std::max(1, (int)std::ceil(std::sqrt((double)maxd2)));
    std::vector<float> sigf(h->P);
    std::vector<int> levbin(h->P);
    std::vector<double> logsig(h->P);
    for (int l = 0; l < h->P; ++l) {
        sigf[l] = (float)sig[l];
        logsig[l] = std::log(sig[l]);
    }
    h->log_lo = logsig[0];
    h->log_hi = logsig[h->P - 1];
    for (int l = 0; l < h->P; ++l) {
        if (c.hist_mode == DOG_HIST_LADDER) {
            levbin[l] = l;
        } else if (h->geom && h->P >= 2) {
            levbin[l] = std::min(c.nbins - 1, (int)(((long long)c.nbins * l) / (h->P - 1)));
        } else {
            const double span = h->log_hi - h->log_lo;
            const double t = (h->P >= 2 && span > 0.0) ? (logsig[l] - h->log_lo) / span : 0.0;
            double fb = std::floor((double)c.nbins * t);
            fb = std::min(std::max(fb, 0.0), (double)(c.nbins - 1));
            levbin[l] = (int)fb;
        }
    }

    // ---- device memory
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(dalloc(&h->d_w, h->w_total));
    ok(dalloc(&h->d_c, cf.size()));
    ok(dalloc(&h->d_sig64, h->P));
    ok(dalloc(&h->d_d2thr, d2.size()));
    ok(dalloc(&h->d_sigf, h->P));
    ok(dalloc(&h->d_levbin, h->P));
    ok(dalloc(&h->d_logsig, h->P));
    h->cand_cap = c.blob_cap;
    h->pend_cap = c.blob_cap;
    ok(dalloc(&h->d_cand, h->cand_cap));
    ok(dalloc(&h->d_counts, 8));
    ok(dalloc(&h->d_pend, h->pend_cap));
    ok(dalloc(&h->d_state, h->cand_cap));
    ok(dalloc(&h->d_target, h->cand_cap));
    ok(dalloc(&h->d_order, h->cand_cap));
    ok(dalloc(&h->d_status, 1));
    ok(dalloc(&h->d_shist, STRETCH_BINS));
    ok(dalloc(&h->d_slohi, 2));
    if (e == cudaSuccess) {
        ok(cudaMemcpy(h->d_w, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_c, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_sig64, sig.data(), sizeof(double) * h->P, cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_d2thr, d2.data(), sizeof(int) * d2.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_sigf, sigf.data(), sizeof(float) * h->P, cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_levbin, levbin.data(), sizeof(int) * h->P, cudaMemcpyHostToDevice));
        ok(cudaMemcpy(h->d_logsig, logsig.data(), sizeof(double) * h->P, cudaMemcpyHostToDevice));
        ok(cudaMemset(h->d_counts, 0, sizeof(int) * 8));
        ok(cudaMemset(h->d_status, 0, sizeof(int)));
    }
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return status_from(e);
    }
    b.w = h->d_w;
    b.c = h->d_c;
    b.status = h->d_status;

    *out = h;
    return DOG_OK;
}

void dog_destroy(dog_t* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    dogk::soft_free(h);
    dogk::fft_free(h->fft);
    free_all(h);
    delete h;
}

int dog_ladder(const dog_t* h, int32_t* K, double* sigmas, int32_t* radii, double* norm) {
    if (!h) return DOG_ERR_INVALID;
    if (K) *K = h->K;
    for (int i = 0; i < h->K; ++i) {
        if (sigmas) sigmas[i] = h->sig[i];
        if (radii) radii[i] = h->rad[i];
    }
    if (norm)
        for (int i = 0; i < h->P; ++i) norm[i] = h->norm[i];
    return DOG_OK;
}

int dog_set_tiling(dog_t* h, int32_t band_rows, int32_t ctas_per_sm) {
    if (!h || band_rows < 0 || (band_rows % MB) != 0 || ctas_per_sm < 1 || ctas_per_sm > 4)
        return DOG_ERR_INVALID;
    h->band = band_rows;
    h->ctas_per_sm = ctas_per_sm;
    return DOG_OK;
}

int dog_set_producer_warps(dog_t* h, int32_t n) {
    if (!h || !(n == 0 || n == 8 || n == 12)) return DOG_ERR_INVALID;
    assign_levels(h, n == 0 ? default_producer_warps(h) : n);
    return DOG_OK;
}

int dog_get_producer_warps(const dog_t* h) { return h ? h->base.nw : DOG_ERR_INVALID; }

// The contrast stretch applies to 12-bit frames when the handle's stretch_sat
// is set (frames of more than 2^31 pixels are not supported then).
static bool stretches(const dog_handle* h, int dtype) {
    return h->cfg.stretch_sat > 0.0 && dtype == DOG_DTYPE_U16;
}

static int check_frame(const dog_handle* h, const void* img, int dtype, int H, int W, int pitch) {
    if (!img || H < 1 || W < 1 || pitch < W) return DOG_ERR_INVALID;
    if (dtype != DOG_DTYPE_F32 && dtype != DOG_DTYPE_U16) return DOG_ERR_INVALID;
    if (H > 65535 || W > 65535) return DOG_ERR_UNSUPPORTED;
    if (stretches(h, dtype) && (long long)H * W >= (1LL << 31)) return DOG_ERR_UNSUPPORTED;
    return DOG_OK;
}

// Limits of a single 12-bit frame into the handle's workspace.
static cudaError_t single_limits(dog_handle* h, const void* img, int H, int W, int pitch, cudaStream_t s) {
    return launch_stretch_limits(nullptr, 1, static_cast<const uint16_t*>(img), H, W, pitch, h->cfg.stretch_sat,
                                 h->num_sms, h->d_shist, h->d_slohi, s);
}

static FusedParams frame_params(const dog_handle* h, const void* img, int dtype, int H, int W, int pitch) {
    FusedParams p = h->base;
    p.img = img;
    p.dtype = stretches(h, dtype) ? DTYPE_U16_STRETCH : dtype;
    p.lohi = h->d_slohi;
    p.H = H;
    p.W = W;
    p.pitch = pitch;
    p.band = (h->band > 0 && h->band < H) ? h->band : ((H + MB - 1) / MB) * MB;
    p.n_strips = (W + TX - 1) / TX;
    p.n_bands = (H + p.band - 1) / p.band;
    p.frames = nullptr;
    return p;
}

static ResolveParams resolve_params(const dog_handle* h, const FusedParams& f) {
    ResolveParams r{};
    r.pend = f.pend;
    r.pend_count = f.pend_count;
    r.pend_cap = f.pend_cap;
    r.frames = nullptr;
    r.img = f.img;
    r.dtype = f.dtype;
    r.lohi = f.lohi;
    r.H = f.H;
    r.W = f.W;
    r.pitch = f.pitch;
    r.K = h->K;
    r.P = h->P;
    r.w = f.w;
    r.c = f.c;
    for (int i = 0; i < h->K; ++i) {
        r.woff[i] = h->woff[i];
        r.r[i] = h->rad[i];
    }
    r.blobs = f.blobs;
    r.cap = f.cap;
    r.count = f.count;
    r.status = h->d_status;
    return r;
}

// The FFT backend's workspace, built on first use from the handle's kernels.
static int fft_ws(dog_handle* h) {
    if (h->fft) return DOG_OK;
    std::vector<std::vector<double>> w(h->K);
    for (int i = 0; i < h->K; ++i) {
        const int r = h->rad[i];
        double z = 0.0;
        for (int j = -r; j <= r; ++j) z += std::exp(-(double)j * j / (2.0 * h->sig[i] * h->sig[i]));
        for (int j = -r; j <= r; ++j) w[i].push_back(std::exp(-(double)j * j / (2.0 * h->sig[i] * h->sig[i])) / z);
    }
    return fft_create(&h->fft, h->cfg.max_h, h->cfg.max_w, h->K, h->R, w);
}

int dog_candidates(dog_t* h, const void* d_img, int32_t dtype, int32_t H, int32_t W, int32_t pitch,
                   dog_blob* d_blobs, int32_t cap, int32_t* d_count, void* stream) {
    if (!h || !d_blobs || !d_count || cap < 0) return DOG_ERR_INVALID;
    int st = check_frame(h, d_img, dtype, H, W, pitch);
    if (st != DOG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    FusedParams p = frame_params(h, d_img, dtype, H, W, pitch);
    if (h->cfg.backend == DOG_BACKEND_FFT) {
        if (H > h->cfg.max_h || W > h->cfg.max_w) return DOG_ERR_INVALID;
        st = fft_ws(h);
        if (st != DOG_OK) return st;
        if (p.dtype == DTYPE_U16_STRETCH) DOG_CUDA(single_limits(h, d_img, H, W, pitch, s));
        return fft_run(h->fft, d_img, p.dtype, H, W, pitch, h->d_slohi, h->P, h->d_c, (float)h->cfg.threshold,
                       MODE_CANDIDATES, d_blobs, cap, d_count, nullptr, h->d_status, s);
    }
    p.mode = MODE_CANDIDATES;
    p.blobs = d_blobs;
    p.cap = cap;
    p.count = d_count;
    p.pend = h->d_pend;
    p.pend_cap = h->pend_cap;
    p.pend_count = h->d_counts + 1;
    DOG_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    DOG_CUDA(cudaMemsetAsync(h->d_counts + 1, 0, sizeof(int), s));
    if (p.dtype == DTYPE_U16_STRETCH) DOG_CUDA(single_limits(h, d_img, H, W, pitch, s));
    DOG_CUDA(timed_fused(h, p, p.n_strips * p.n_bands, s));
    ResolveParams r = resolve_params(h, p);
    DOG_CUDA(launch_resolve(r, h->pend_cap, s));
    return DOG_OK;
}

int dog_debug_dog(dog_t* h, const void* d_img, int32_t dtype, int32_t H, int32_t W, int32_t pitch,
                  float* d_dog, void* stream) {
    if (!h || !d_dog) return DOG_ERR_INVALID;
    int st = check_frame(h, d_img, dtype, H, W, pitch);
    if (st != DOG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    FusedParams p = frame_params(h, d_img, dtype, H, W, pitch);
    if (h->cfg.backend == DOG_BACKEND_FFT) {
        if (H > h->cfg.max_h || W > h->cfg.max_w) return DOG_ERR_INVALID;
        st = fft_ws(h);
        if (st != DOG_OK) return st;
        if (p.dtype == DTYPE_U16_STRETCH) DOG_CUDA(single_limits(h, d_img, H, W, pitch, s));
        return fft_run(h->fft, d_img, p.dtype, H, W, pitch, h->d_slohi, h->P, h->d_c, (float)h->cfg.threshold,
                       MODE_DUMP, nullptr, 0, nullptr, d_dog, h->d_status, s);
    }
    p.mode = MODE_DUMP;
    p.dump = d_dog;
    if (p.dtype == DTYPE_U16_STRETCH) DOG_CUDA(single_limits(h, d_img, H, W, pitch, s));
    DOG_CUDA(timed_fused(h, p, p.n_strips * p.n_bands, s));
    return DOG_OK;
}

static PruneParams prune_params(const dog_handle* h) {
    PruneParams q{};
    q.P = h->P;
    q.sig = h->d_sig64;
    q.d2thr = h->d_d2thr;
    q.cell = h->cell;
    q.mode = h->cfg.prune;
    q.status = h->d_status;
    return q;
}

int dog_prune(dog_t* h, const dog_blob* d_cand, const int32_t* d_count, int32_t cap_in, int32_t H,
              int32_t W, dog_blob* d_out, int32_t cap_out, int32_t* d_nout, void* stream) {
    if (!h || !d_cand || !d_count || !d_out || !d_nout || cap_in < 0 || cap_out < 0 || H < 1 || W < 1)
        return DOG_ERR_INVALID;
    if (cap_in > h->cand_cap) return DOG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    PruneParams q = prune_params(h);
    q.cand = d_cand;
    q.cand_count = d_count;
    q.cap_in = cap_in;
    q.n_frames = 1;
    q.H = H;
    q.W = W;
    q.state = h->d_state;
    q.target = h->d_target;
    q.order = h->d_order;
    q.out = d_out;
    q.cap_out = cap_out;
    q.out_count = d_nout;
    DOG_CUDA(launch_prune(q, s));
    return DOG_OK;
}

static HistParams hist_params(const dog_handle* h) {
    HistParams q{};
    q.P = h->P;
    q.nbins = h->cfg.nbins;
    q.mode = h->cfg.hist_mode;
    q.sig_f = h->d_sigf;
    q.level_bin = h->d_levbin;
    q.log_sig = h->d_logsig;
    q.log_lo = h->log_lo;
    q.log_hi = h->log_hi;
    return q;
}

static int hist_bins(const dog_handle* h) {
    return h->cfg.hist_mode == DOG_HIST_LADDER ? h->P : h->cfg.nbins;
}

int dog_volume_hist(dog_t* h, const dog_blob* d_blobs, const int32_t* d_count, int32_t cap,
                    uint32_t* d_hist, double* d_hist_vol, void* stream) {
    if (!h || !d_blobs || !d_count || !d_hist || cap < 0) return DOG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const int nb = hist_bins(h);
    DOG_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * nb, s));
    if (d_hist_vol) DOG_CUDA(cudaMemsetAsync(d_hist_vol, 0, sizeof(double) * nb, s));
    HistParams q = hist_params(h);
    q.blobs = d_blobs;
    q.count = d_count;
    q.cap = cap;
    q.n_frames = 1;
    q.hist = d_hist;
    q.vol = d_hist_vol;
    DOG_CUDA(launch_hist(q, s));
    return DOG_OK;
}

int dog_detect(dog_t* h, const void* d_img, int32_t dtype, int32_t H, int32_t W, int32_t pitch,
               dog_blob* d_blobs, int32_t cap, int32_t* d_count, uint32_t* d_hist, double* d_hist_vol,
               void* stream) {
    if (!h || !d_blobs || !d_count || cap < 0) return DOG_ERR_INVALID;
    int st = dog_candidates(h, d_img, dtype, H, W, pitch, h->d_cand, h->cand_cap, h->d_counts + 0, stream);
    if (st != DOG_OK) return st;
    // pruning, with the histogram of the pruned blobs computed by the same
    // kernel (one launch fewer on the single-frame latency path)
    cudaStream_t s = (cudaStream_t)stream;
    PruneParams q = prune_params(h);
    q.cand = h->d_cand;
    q.cand_count = h->d_counts + 0;
    q.cap_in = h->cand_cap;
    q.n_frames = 1;
    q.H = H;
    q.W = W;
    q.state = h->d_state;
    q.target = h->d_target;
    q.order = h->d_order;
    q.out = d_blobs;
    q.cap_out = cap;
    q.out_count = d_count;
    if (d_hist) {
        q.hist = hist_params(h);
        q.hist.hist = d_hist;
        q.hist.vol = d_hist_vol;
    }
    DOG_CUDA(launch_prune(q, s));
    return DOG_OK;
}

static int grow_batch(dog_handle* h, int n) {
    if (n <= h->batch_cap) return DOG_OK;
    cudaDeviceSynchronize();
    void* olds[] = {h->d_desc, h->d_cand_off, h->d_out_off, h->d_hw, h->d_ntiles, h->d_bcand,
                    h->d_bstate, h->d_btarget, h->d_border, h->d_bcounts, h->d_bpend, h->d_bshist, h->d_bslohi};
    for (void* p : olds)
        if (p) cudaFree(p);
    h->d_desc = nullptr; h->d_cand_off = nullptr; h->d_out_off = nullptr; h->d_hw = nullptr;
    h->d_ntiles = nullptr; h->d_bcand = nullptr; h->d_bstate = nullptr; h->d_btarget = nullptr;
    h->d_border = nullptr; h->d_bcounts = nullptr; h->d_bpend = nullptr; h->d_bshist = nullptr;
    h->d_bslohi = nullptr;
    h->batch_cap = 0;
    const size_t nc = (size_t)n * h->cand_cap;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(dalloc(&h->d_desc, n));
    ok(dalloc(&h->d_cand_off, n));
    ok(dalloc(&h->d_out_off, n));
    ok(dalloc(&h->d_hw, 2 * n));
    ok(dalloc(&h->d_ntiles, 1));
    ok(dalloc(&h->d_bcand, nc));
    ok(dalloc(&h->d_bstate, nc));
    ok(dalloc(&h->d_btarget, nc));
    ok(dalloc(&h->d_border, nc));
    ok(dalloc(&h->d_bcounts, n + 4));
    h->bpend_cap = (int)std::min<size_t>(nc, (size_t)1 << 26);
    ok(dalloc(&h->d_bpend, h->bpend_cap));
    ok(dalloc(&h->d_bshist, (size_t)n * STRETCH_BINS));
    ok(dalloc(&h->d_bslohi, 2 * (size_t)n));
    if (e == cudaSuccess) ok(cudaMemset(h->d_bcounts, 0, sizeof(int) * (n + 4)));
    if (e != cudaSuccess) return status_from(e);
    h->batch_cap = n;
    return DOG_OK;
}

int dog_detect_batched(dog_t* h, const dog_frame* d_frames, int32_t n, int32_t max_h, int32_t max_w,
                       dog_blob* d_blobs, int32_t* d_counts, uint32_t* d_hists, void* stream) {
    if (!h || !d_frames || n < 1 || !d_blobs || !d_counts || max_h < 1 || max_w < 1) return DOG_ERR_INVALID;
    if (h->cfg.backend != DOG_BACKEND_DIRECT || !h->direct_ok) return DOG_ERR_UNSUPPORTED;
    const bool stretch = h->cfg.stretch_sat > 0.0;
    if (stretch && (long long)max_h * max_w >= (1LL << 31)) return DOG_ERR_UNSUPPORTED;
    int st = grow_batch(h, n);
    if (st != DOG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const int band = (h->band > 0) ? h->band : 0;
    // per-frame descriptors, candidate/output offsets and the tile prefix sum
    const int grid = h->num_sms * h->ctas_per_sm;
    // contrast-stretch limits of the batch's 12-bit frames
    if (stretch)
        DOG_CUDA(launch_stretch_limits(d_frames, n, nullptr, 0, 0, 0, h->cfg.stretch_sat, h->num_sms, h->d_bshist,
                                       h->d_bslohi, s));
    DOG_CUDA(launch_batch_prep(d_frames, n, band, grid, h->cand_cap, stretch, h->d_desc, h->d_cand_off,
                               h->d_out_off, h->d_hw, h->d_ntiles, s));
    // fixed slots: the persistent kernel's work and completion counters are
    // zero between launches (the last CTA resets them), whatever n was
    int* tile_counter = h->d_bcounts + 0;
    int* done_counter = h->d_bcounts + 1;
    int* pend_count = h->d_bcounts + 2;
    int* cand_counts = h->d_bcounts + 3;          // n
    DOG_CUDA(cudaMemsetAsync(pend_count, 0, sizeof(int) * (n + 1), s));
    FusedParams p = h->base;
    p.frames = h->d_desc;
    p.n_frames = n;
    p.n_tiles = 0;   // read from device
    p.band = band;
    p.tile_counter = tile_counter;
    p.done_counter = done_counter;
    p.mode = MODE_CANDIDATES;
    p.blobs = h->d_bcand;
    p.cap = h->cand_cap;
    p.count = cand_counts;
    p.pend = h->d_bpend;
    p.pend_cap = h->bpend_cap;
    p.pend_count = pend_count;
    p.ntiles_dev = h->d_ntiles;
    p.lohi = h->d_bslohi;
    DOG_CUDA(timed_fused(h, p, grid, s));
    ResolveParams r = resolve_params(h, p);
    r.frames = h->d_desc;
    r.blobs = h->d_bcand;
    r.cap = h->cand_cap;
    r.count = cand_counts;
    DOG_CUDA(launch_resolve(r, std::min(h->bpend_cap, 152 * 64), s));
    PruneParams q = prune_params(h);
    q.cand = h->d_bcand;
    q.cand_count = cand_counts;
    q.cap_in = h->cand_cap;
    q.cand_off = h->d_cand_off;
    q.n_frames = n;
    q.frame_hw = h->d_hw;
    q.H = max_h;
    q.W = max_w;
    q.state = h->d_bstate;
    q.target = h->d_btarget;
    q.order = h->d_border;
    q.out = d_blobs;
    q.cap_out = h->cand_cap;
    q.out_off = h->d_out_off;
    q.out_count = d_counts;
    if (d_hists) {   // each frame's histogram from its pruning CTA
        q.hist = hist_params(h);
        q.hist.hist = d_hists;
        q.hist.vol = nullptr;
    }
    DOG_CUDA(launch_prune(q, s));
    return DOG_OK;
}

int dog_soft_hist(dog_t* h, const float* d_img, int32_t H, int32_t W, int32_t pitch, const float* d_sigmas,
                  float* d_soft_hist, void* stream) {
    if (!h || !d_sigmas || !d_soft_hist) return DOG_ERR_INVALID;
    if (!h->direct_ok) return DOG_ERR_UNSUPPORTED;
    int st = check_frame(h, d_img, DOG_DTYPE_F32, H, W, pitch);
    if (st != DOG_OK) return st;
    h->last = (cudaStream_t)stream;
    return soft_forward(h, d_img, H, W, pitch, d_sigmas, d_soft_hist, nullptr, 0, nullptr, (cudaStream_t)stream);
}

int dog_soft_hist_rec(dog_t* h, const float* d_img, int32_t H, int32_t W, int32_t pitch, const float* d_sigmas,
                      float* d_soft_hist, dog_soft_max* d_max, int32_t cap, int32_t* d_count, void* stream) {
    if (!h || !d_sigmas || !d_soft_hist || !d_max || !d_count || cap < 1) return DOG_ERR_INVALID;
    if (!h->direct_ok) return DOG_ERR_UNSUPPORTED;
    int st = check_frame(h, d_img, DOG_DTYPE_F32, H, W, pitch);
    if (st != DOG_OK) return st;
    h->last = (cudaStream_t)stream;
    return soft_forward(h, d_img, H, W, pitch, d_sigmas, d_soft_hist, d_max, cap, d_count, (cudaStream_t)stream);
}

int dog_backward_rec(dog_t* h, const float* d_img, int32_t H, int32_t W, int32_t pitch, const float* d_sigmas,
                     const dog_soft_max* d_max, const int32_t* d_count, int32_t cap, const float* d_grad_hist,
                     float* d_grad_img, float* d_grad_sigmas, void* stream) {
    if (!h || !d_sigmas || !d_max || !d_count || cap < 1 || !d_grad_hist || !d_grad_img || !d_grad_sigmas)
        return DOG_ERR_INVALID;
    if (!h->direct_ok) return DOG_ERR_UNSUPPORTED;
    int st = check_frame(h, d_img, DOG_DTYPE_F32, H, W, pitch);
    if (st != DOG_OK) return st;
    h->last = (cudaStream_t)stream;
    return soft_backward_rec(h, d_img, H, W, pitch, d_sigmas, d_max, d_count, cap, d_grad_hist, d_grad_img,
                             d_grad_sigmas, (cudaStream_t)stream);
}

int dog_backward(dog_t* h, const float* d_img, int32_t H, int32_t W, int32_t pitch, const float* d_sigmas,
                 const float* d_grad_hist, float* d_grad_img, float* d_grad_sigmas, void* stream) {
    if (!h || !d_sigmas || !d_grad_hist || !d_grad_img || !d_grad_sigmas) return DOG_ERR_INVALID;
    if (!h->direct_ok) return DOG_ERR_UNSUPPORTED;
    int st = check_frame(h, d_img, DOG_DTYPE_F32, H, W, pitch);
    if (st != DOG_OK) return st;
    h->last = (cudaStream_t)stream;
    return soft_backward(h, d_img, H, W, pitch, d_sigmas, d_grad_hist, d_grad_img, d_grad_sigmas,
                         (cudaStream_t)stream);
}

int dog_ring_hist_push(const uint32_t* d_hist, int32_t nbins, uint32_t* d_ring, int32_t window,
                       uint32_t* d_sum, int32_t* d_head, void* stream) {
    if (!d_hist || !d_ring || !d_sum || !d_head || nbins < 1 || window < 1) return DOG_ERR_INVALID;
    return status_from(launch_ring_push(d_hist, nbins, d_ring, window, d_sum, d_head, (cudaStream_t)stream));
}

int dog_ring_hist_push_batched(const uint32_t* d_hists, const int32_t* d_stream_ids, int32_t n, int32_t nbins,
                               int32_t n_streams, uint32_t* d_rings, int32_t window, uint32_t* d_sums,
                               int32_t* d_heads, void* stream) {
    if (!d_hists || !d_stream_ids || !d_rings || !d_sums || !d_heads || n < 0 || nbins < 1 || n_streams < 1 ||
        window < 1)
        return DOG_ERR_INVALID;
    if (n == 0) return DOG_OK;
    return status_from(launch_ring_push_batched(d_hists, d_stream_ids, n, nbins, n_streams, d_rings, window,
                                                d_sums, d_heads, (cudaStream_t)stream));
}

int dog_profile_enable(dog_t* h, int32_t enable) {
    if (!h) return DOG_ERR_INVALID;
    h->prof = enable != 0;
    return DOG_OK;
}

int dog_profile_read(dog_t* h, double* h_ms, int32_t* h_launches) {
    if (!h || !h_ms || !h_launches) return DOG_ERR_INVALID;
    double total = 0.0;
    for (int i = 0; i < h->ev_used; ++i) {
        if (cudaEventSynchronize(h->ev[2 * i + 1]) != cudaSuccess) return DOG_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess) return DOG_ERR_CUDA;
        total += ms;
    }
    *h_ms = total;
    *h_launches = h->ev_used;
    h->ev_used = 0;
    return DOG_OK;
}

int dog_get_status(dog_t* h, int32_t* h_status) {
    if (!h || !h_status) return DOG_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(h->last);
    if (e != cudaSuccess) return DOG_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DOG_ERR_CUDA;
    if (cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) return DOG_ERR_CUDA;
    *h_status = v;
    return DOG_OK;
}

int dog_test_fail_alloc(int32_t after) {
    if (after < -1) return DOG_ERR_INVALID;
    g_fail_after.store(after);
    return DOG_OK;
}

const char* dog_status_string(int status) {
    switch (status) {
        case DOG_OK: return "ok";
        case DOG_ERR_INVALID: return "invalid argument";
        case DOG_ERR_NOMEM: return "out of memory";
        case DOG_ERR_CUDA: return "CUDA error";
        case DOG_ERR_CAPACITY: return "blob list capacity exceeded";
        case DOG_ERR_TIMEOUT: return "device wait timed out";
        case DOG_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

}  // extern "C"
