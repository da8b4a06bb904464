// Differentiable soft blob-volume histogram and its backward pass (sm_103a).
//
// Not in the paper: a smooth relaxation of the volume histogram of Sec. 4 so
// that the sigma ladder can be tuned by gradient descent towards a steering
// objective.  Over the hard 3x3x3 local maxima v of D (no threshold),
//   H_b = sum_v s_v kappa_b(t_l),   s_v = sigmoid((D_v - thr) / T),
// t_l the normalised log volume of plane l against the handle's ladder ends
// and kappa_b a triangular weight one bin wide.  With the mask and radii
// held fixed, for dloss/dH = gH:
//   G_v = (sum_b gH_b kappa_b(t_l)) s_v (1 - s_v) / T          (dloss/dD_v)
//   A_i = c_i G_i - c_{i-1} G_{i-1}                             (dloss/dL_i)
//   dloss/dI = sum_i B_i^T A_i,     B_i = row blur o column blur (reflect)
//   dloss/dsigma_i = <B_y^T A_i, B_x' I> + <B_y'^T A_i, B_x I>  (kernel shape)
//                  + dloss/dc terms + dloss/dt terms.
// Two backward paths.  From a record of the forward's maxima (soft forward
// with `rec`): A is scattered from the list, and the kernel-shape term is
// evaluated at the maxima as sum_v A_i(v) dL_i/dsigma_i(v) (the same sum,
// since A_i vanishes elsewhere); no blur level is formed.  Without a record:
// the fused kernel (MODE_BWD) recomputes the L_i and writes A densely, and
// the kernel-shape term is the two inner products above.  Both then run the
// adjoint blurs, which gather through the reflect fold-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dog_internal.cuh"

namespace dogk {

const FusedParams& handle_base(const dog_handle* h);
int handle_K(const dog_handle* h);
int handle_P(const dog_handle* h);
const std::vector<int>& handle_radii(const dog_handle* h);
const std::vector<double>& handle_sigmas(const dog_handle* h);
const dog_config& handle_cfg(const dog_handle* h);
int handle_band(const dog_handle* h);
int* handle_status(dog_handle* h);
void*& handle_soft_ws(dog_handle* h);
cudaError_t timed_fused(dog_handle* h, const FusedParams& p, int grid, cudaStream_t s);

struct SoftWS {
    int H = 0, W = 0;
    float* w = nullptr;       // half kernels from the device sigmas
    float* dw = nullptr;      // their derivative wrt sigma
    float* c = nullptr;       // P coefficients then P sigmas
    float* kappa = nullptr;   // P x nbins
    float* dkappa = nullptr;  // P x nbins
    Pending* pend = nullptr;
    int pend_cap = 0;
    int* counts = nullptr;
    float* A = nullptr;       // K x H x W
    float* Y = nullptr;       // K x H x W
    float* Yd = nullptr;      // K x H x W
    double* acc = nullptr;    // dc (P), dt (P), dw (K)
    float* last_sig = nullptr;   // the sigmas the tables were last built from (NaN: none)
    int* big = nullptr;          // wide-window maxima queued by the sigma kernel
    int* big_count = nullptr;
    int big_cap = 0;
};

void soft_free(dog_handle* h) {
    SoftWS* ws = static_cast<SoftWS*>(handle_soft_ws(h));
    if (!ws) return;
    void* ptrs[] = {ws->w, ws->dw, ws->c, ws->kappa, ws->dkappa, ws->pend, ws->counts, ws->A, ws->Y, ws->Yd, ws->acc,
                    ws->last_sig, ws->big, ws->big_count};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete ws;
    handle_soft_ws(h) = nullptr;
}

static int soft_ws(dog_handle* h, int H, int W, SoftWS** out) {
    SoftWS* ws = static_cast<SoftWS*>(handle_soft_ws(h));
    if (ws && ws->H >= H && ws->W >= W) { *out = ws; return DOG_OK; }
    if (ws) { cudaDeviceSynchronize(); soft_free(h); }
    ws = new SoftWS();
    handle_soft_ws(h) = ws;
    const FusedParams& b = handle_base(h);
    const int K = b.K, P = b.P, nb = handle_cfg(h).nbins;
    const size_t plane = (size_t)H * W;
    const int strips = (W + TX - 1) / TX;
    ws->pend_cap = (int)std::min<size_t>((size_t)2 * strips * P * H + 1024, (size_t)1 << 28);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(cudaMalloc(&ws->w, sizeof(float) * b.w_total));
    ok(cudaMalloc(&ws->dw, sizeof(float) * b.w_total));
    ok(cudaMalloc(&ws->c, sizeof(float) * 2 * P));
    ok(cudaMalloc(&ws->kappa, sizeof(float) * P * nb));
    ok(cudaMalloc(&ws->dkappa, sizeof(float) * P * nb));
    ok(cudaMalloc(&ws->pend, sizeof(Pending) * ws->pend_cap));
    ok(cudaMalloc(&ws->counts, sizeof(int) * 4));
    ok(cudaMalloc(&ws->A, sizeof(float) * plane * K));
    ok(cudaMalloc(&ws->Y, sizeof(float) * plane * K));
    ok(cudaMalloc(&ws->Yd, sizeof(float) * plane * K));
    ok(cudaMalloc(&ws->acc, sizeof(double) * (2 * P + K)));
    ok(cudaMalloc(&ws->last_sig, sizeof(float) * K));
    ws->big_cap = 1 << 16;
    ok(cudaMalloc(&ws->big, sizeof(int) * ws->big_cap));
    ok(cudaMalloc(&ws->big_count, sizeof(int)));
    if (e == cudaSuccess) ok(cudaMemset(ws->last_sig, 0xff, sizeof(float) * K));   // NaN: tables not built
    if (e != cudaSuccess) {
        soft_free(h);
        return e == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA;
    }
    ws->H = H;
    ws->W = W;
    *out = ws;
    return DOG_OK;
}

// ---------------------------------------------------------------------------
struct SoftPrep {
    const float* sig;
    int K, P, nbins, norm;
    int r[MAX_LEVELS];
    int woff[MAX_LEVELS];
    int tpad[MAX_LEVELS];
    int hoff[MAX_LEVELS];    // the horizontal pass's copy of the taps
    double lref0, lrefP;   // ln sigma of the reference ladder's first / last DoG plane
    float* w;
    float* dw;
    float* c;
    float* kappa;
    float* dkappa;
    float* last_sig;
};

// Tap, coefficient and bin-weight tables of the device sigmas.  Skipped when
// the sigmas equal those the tables were last built from (a batch of frames
// at one ladder builds them once); last_sig is NaN after allocation.
constexpr int PREP_THREADS = 512;
__global__ void __launch_bounds__(PREP_THREADS) soft_prep_kernel(const __grid_constant__ SoftPrep p) {
    bool changed = false;
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) changed |= !(p.sig[i] == p.last_sig[i]);
    if (!__syncthreads_or(changed)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < p.K; i += PREP_THREADS / 32) {
        const double s = (double)p.sig[i];
        const int r = p.r[i];
        double z = 0.0, m2 = 0.0;
        for (int j = -r + lane; j <= r; j += 32) {
            const double e = exp(-(double)j * j / (2.0 * s * s));
            z += e;
            m2 += e * (double)j * j;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            z += __shfl_xor_sync(0xffffffffu, z, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        m2 /= z;
        // full taps t = 0..2r (offset t - r), zero-padded to tpad
        for (int t = lane; t < p.tpad[i]; t += 32) {
            const int j = t - r;
            float wv = 0.0f, dv = 0.0f;
            if (t <= 2 * r) {
                const double wj = exp(-(double)j * j / (2.0 * s * s)) / z;
                wv = (float)wj;
                dv = (float)(wj * ((double)j * j - m2) / (s * s * s));
            }
            p.w[p.woff[i] + t] = wv;
            p.dw[p.woff[i] + t] = dv;
            p.w[p.hoff[i] + t] = wv;
        }
    }
    for (int l = threadIdx.x; l < p.P; l += blockDim.x) {
        const double s0 = (double)p.sig[l], s1 = (double)p.sig[l + 1];
        p.c[l] = (float)(p.norm == DOG_NORM_PAPER ? s0 : s0 / (s1 - s0));
        p.c[p.P + l] = (float)s0;
        const double t = (log(s0) - p.lref0) / (p.lrefP - p.lref0);
        const double lo = 0.5 / p.nbins, hi = 1.0 - 0.5 / p.nbins;
        const bool clamped = (t < lo) || (t > hi);
        const double tc = fmin(fmax(t, lo), hi);
        for (int b = 0; b < p.nbins; ++b) {
            const double u = (double)p.nbins * tc - ((double)b + 0.5);
            const double a = fabs(u);
            p.kappa[l * p.nbins + b] = a < 1.0 ? (float)(1.0 - a) : 0.0f;
            const double sg = u > 0.0 ? 1.0 : (u < 0.0 ? -1.0 : 0.0);
            p.dkappa[l * p.nbins + b] = (a < 1.0 && !clamped) ? (float)(-(double)p.nbins * sg) : 0.0f;
        }
    }
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) p.last_sig[i] = p.sig[i];
}

static SoftPrep prep_params(dog_handle* h, SoftWS* ws, const float* sig) {
    const FusedParams& b = handle_base(h);
    const std::vector<double>& ref = handle_sigmas(h);
    SoftPrep q{};
    q.sig = sig;
    q.K = b.K;
    q.P = b.P;
    q.nbins = handle_cfg(h).nbins;
    q.norm = handle_cfg(h).norm;
    for (int i = 0; i < b.K; ++i) {
        q.r[i] = b.lv[i].r;
        q.woff[i] = b.lv[i].woff;
        q.tpad[i] = b.lv[i].tpad;
        q.hoff[i] = b.lv[i].hoff;
    }
    q.lref0 = std::log(ref[0]);
    q.lrefP = std::log(ref[b.P - 1]);
    q.w = ws->w;
    q.dw = ws->dw;
    q.c = ws->c;
    q.kappa = ws->kappa;
    q.dkappa = ws->dkappa;
    q.last_sig = ws->last_sig;
    return q;
}

static FusedParams soft_fused(dog_handle* h, SoftWS* ws, const float* img, int H, int W, int pitch, int mode) {
    FusedParams p = handle_base(h);
    p.img = img;
    p.dtype = DOG_DTYPE_F32;
    p.H = H;
    p.W = W;
    p.pitch = pitch;
    const int band = handle_band(h);
    p.band = (band > 0 && band < H) ? band : ((H + MB - 1) / MB) * MB;
    // overlapping strips (32 columns stepping by 30): every local maximum is
    // settled inside the fused kernel, so no strip-edge resolve follows (the
    // soft modes keep every maximum, thousands per frame at strip edges)
    p.overlap = 1;
    p.n_strips = (W + TX - 2 - 1) / (TX - 2);
    p.n_bands = (H + p.band - 1) / p.band;
    p.frames = nullptr;
    p.mode = mode;
    p.w = ws->w;
    p.c = ws->c;
    p.pend = ws->pend;
    p.pend_cap = ws->pend_cap;
    p.pend_count = ws->counts;
    p.kappa = ws->kappa;
    p.dkappa = ws->dkappa;
    p.nbins = handle_cfg(h).nbins;
    p.inv_T = (float)(1.0 / handle_cfg(h).soft_T);
    p.status = handle_status(h);
    return p;
}

#define SOFT_CUDA(x)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA; \
    } while (0)

int soft_forward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig, float* out,
                 dog_soft_max* rec, int rec_cap, int* rec_count, cudaStream_t s) {
    SoftWS* ws = nullptr;
    int st = soft_ws(h, H, W, &ws);
    if (st != DOG_OK) return st;
    SoftPrep q = prep_params(h, ws, sig);
    soft_prep_kernel<<<1, PREP_THREADS, 0, s>>>(q);
    SOFT_CUDA(cudaGetLastError());
    SOFT_CUDA(cudaMemsetAsync(ws->counts, 0, sizeof(int) * 4, s));
    FusedParams p = soft_fused(h, ws, img, H, W, pitch, MODE_SOFT);
    p.soft_out = out;
    if (rec != nullptr) {
        SOFT_CUDA(cudaMemsetAsync(rec_count, 0, sizeof(int), s));
        p.rec = rec;
        p.rec_cap = rec_cap;
        p.rec_count = rec_count;
    }
    SOFT_CUDA(timed_fused(h, p, p.n_strips * p.n_bands, s));
    return DOG_OK;
}

// ---------------------------------------------------------------------------
// Reflected part of the 1-D adjoint of a reflect-boundary correlation with the
// symmetric full kernel w[0..2r] (w[r + d] weighs offset d), at index m of a
// line of length N with stride `st`.  The adjoint at m sums, over the
// preimages q of m under the reflection that lie within r of the line,
// sum_n w[|q-n|] a[n]; the zero-padded correlation gives the term q = m, and
// this function the others (the reflected copies q = -1-m, 2N-1-m, ...).
__device__ __forceinline__ float adj1d_mirror(const float* __restrict__ a, size_t st, int N, int m,
                                              const float* __restrict__ w, int r) {
    float acc = 0.0f;
    const int per = 2 * N;
    const int fam[2] = {m, per - 1 - m};
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        int q = fam[f];
        const int k = (-r - q) > 0 ? ((-r - q) + per - 1) / per : -((q + r) / per);
        for (q = q + k * per; q <= N - 1 + r; q += per) {
            if (q == m) continue;
            const int nlo = max(0, q - r), nhi = min(N - 1, q + r);
            for (int n = nlo; n <= nhi; ++n) acc = __fmaf_rn(__ldg(w + r + (q - n)), __ldg(a + (size_t)n * st), acc);
        }
    }
    return acc;
}

// Outputs of a line of length N that a reflected preimage reaches (those
// within r of an end): count, and the j-th of them.
__host__ __device__ inline int fold_count(int N, int r) { return N <= 2 * r ? N : 2 * r; }
__host__ __device__ inline int fold_index(int N, int r, int j) { return (N <= 2 * r || j < r) ? j : N - 2 * r + j; }

__device__ __forceinline__ int refl_i(int i, int n) {
    if (i >= 0 && i < n) return i;   // inside: no modulo
    int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m >= n ? p - 1 - m : m;
}

struct AdjParams {
    const float* A;
    float* Y;
    float* Yd;
    const float* img;
    int pitch;
    float* gimg;
    int H, W, K, R;
    const float* w;
    const float* dw;
    int r[MAX_LEVELS];
    int tpad[MAX_LEVELS];
    int woff[MAX_LEVELS];
    double* dw_acc;
};

// Tiled adjoints.  Both kernels of a level, w(t) and dw/dsigma(t), are even
// in t, so away from the frame's edges the adjoint of a blur is the same
// correlation: out(m) = sum_{u < Tpad} k[u] X(m - r + u) over zero-padded taps.
// Eight consecutive outputs per thread are accumulated against a two-window
// register file (8 inputs per block of 8 taps), for two tap sets at once.
// Outputs within r of an edge, where the reflect boundary folds the sums, get
// the reflected preimages' part added afterwards by the fold kernels, one
// thread per such output (adj1d_mirror).
__device__ __forceinline__ void tap_block2(float (&o)[8], float (&od)[8], const float (&A)[8], const float (&B)[8],
                                           const float* __restrict__ w, const float* __restrict__ dw) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const float a = w[u], b = dw[u];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float x = (k + u < 8) ? A[k + u] : B[k + u - 8];
            o[k] = __fmaf_rn(a, x, o[k]);
            od[k] = __fmaf_rn(b, x, od[k]);
        }
    }
}

// out[k] = sum_u w[u] X[(k + u) st], od[k] with dw; u < 8 nb.
__device__ __forceinline__ void corr8x2(const float* __restrict__ X, int st, const float* __restrict__ w,
                                        const float* __restrict__ dw, int nb, float (&o)[8], float (&od)[8]) {
    float A[8], B[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        o[k] = 0.0f;
        od[k] = 0.0f;
        A[k] = X[k * st];
    }
    int j = 0;
    for (;;) {
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = X[(8 * j + 8 + k) * st];
        tap_block2(o, od, A, B, w + 8 * j, dw + 8 * j);
        if (++j == nb) break;
#pragma unroll
        for (int k = 0; k < 8; ++k) A[k] = X[(8 * j + 8 + k) * st];
        tap_block2(o, od, B, A, w + 8 * j, dw + 8 * j);
        if (++j == nb) break;
    }
}

// One tap set: out[k] = sum_u w[u] X[(k + u) st], u < 8 nb.
__device__ __forceinline__ void corr8(const float* __restrict__ X, int st, const float* __restrict__ w, int nb,
                                      float (&o)[8]) {
    float A[8], B[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        o[k] = 0.0f;
        A[k] = X[k * st];
    }
    int j = 0;
    for (;;) {
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = X[(8 * j + 8 + k) * st];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = __fmaf_rn(w[8 * j + u], (k + u < 8) ? A[k + u] : B[k + u - 8], o[k]);
        if (++j == nb) break;
#pragma unroll
        for (int k = 0; k < 8; ++k) A[k] = X[(8 * j + 8 + k) * st];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = __fmaf_rn(w[8 * j + u], (k + u < 8) ? B[k + u] : A[k + u - 8], o[k]);
        if (++j == nb) break;
    }
}

constexpr int ADJ_TM = 64;     // output rows per CTA of the column adjoint

__host__ __device__ inline int adj_y_smem_floats(int tpad_max) { return (ADJ_TM + tpad_max + 8) * 32 + 2 * tpad_max; }

// Column adjoint of level blockIdx.z: Y_i = B_y^T A_i (kernel w_i) and, when
// SIG, Yd_i (dw_i) for the dense sigma gradient; a 32-column x 64-row tile per
// CTA, warp g on rows 8g .. 8g+7, lane = column.
template <bool SIG>
__global__ void __launch_bounds__(256) adj_y_kernel(const __grid_constant__ AdjParams p) {
    extern __shared__ float ysm[];
    const int i = blockIdx.z;
    const int r = p.r[i], tpad = p.tpad[i], nb = tpad >> 3;
    const int x0 = blockIdx.x * 32, m0 = blockIdx.y * ADJ_TM;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int rows = ADJ_TM + tpad + 8;
    float* X = ysm;                  // rows x 32: A rows m0 - r + j, zero outside the frame
    float* ws = ysm + rows * 32;     // tpad
    float* wd = ws + tpad;           // tpad
    const size_t plane = (size_t)p.H * p.W;
    const float* A = p.A + plane * i;
    for (int t = threadIdx.x; t < tpad; t += blockDim.x) {
        ws[t] = p.w[p.woff[i] + t];
        wd[t] = p.dw[p.woff[i] + t];
    }
    const int x = x0 + lane;
    // warp g stages rows g, g + 8, ...; eight loads in flight before the stores
    for (int j0 = g; j0 < rows; j0 += 64) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = j0 + 8 * u, n = m0 - r + j;
            v[u] = (j < rows && n >= 0 && n < p.H && x < p.W) ? A[(size_t)n * p.W + x] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + 8 * u < rows) X[(j0 + 8 * u) * 32 + lane] = v[u];
    }
    __syncthreads();
    float o[8], od[8];
    if (SIG)
        corr8x2(X + 8 * g * 32 + lane, 32, ws, wd, nb, o, od);
    else
        corr8(X + 8 * g * 32 + lane, 32, ws, nb, o);
    if (x >= p.W) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int m = m0 + 8 * g + k;
        if (m >= p.H) break;
        p.Y[plane * i + (size_t)m * p.W + x] = o[k];
        if (SIG) p.Yd[plane * i + (size_t)m * p.W + x] = od[k];
    }
}

// Reflect fold of the column adjoint: rows within r_i of the top or bottom
// edge (blockIdx.y-th of them) of level blockIdx.z, one thread per column.
template <bool SIG>
__global__ void __launch_bounds__(128) adj_y_fold_kernel(const __grid_constant__ AdjParams p) {
    const int i = blockIdx.z, r = p.r[i];
    const int j = blockIdx.y;
    if (j >= fold_count(p.H, r)) return;
    const int m = fold_index(p.H, r, j);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.W) return;
    const size_t plane = (size_t)p.H * p.W;
    const float* A = p.A + plane * i + x;
    const size_t o = plane * i + (size_t)m * p.W + x;
    p.Y[o] += adj1d_mirror(A, p.W, p.H, m, p.w + p.woff[i], r);
    if (SIG) p.Yd[o] += adj1d_mirror(A, p.W, p.H, m, p.dw + p.woff[i], r);
}

// Reflect fold of the row adjoint: one warp per row y, its lanes on the
// columns within R of the left or right edge; sums the reflected preimages'
// part over every level whose radius reaches the column.  When the frame is
// wider than 2R, a level's reflected terms read only the first and last r_i
// values of the row, which the warp first stages in shared memory (one round
// of coalesced loads per level instead of a serial chain of global loads).
constexpr int FOLD_ROWS = 4;   // warps (rows) per CTA
__global__ void __launch_bounds__(32 * FOLD_ROWS) adj_x_fold_kernel(const __grid_constant__ AdjParams p) {
    __shared__ float edge[FOLD_ROWS][2][DOG_MAX_RADIUS];
    const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * FOLD_ROWS + wq;
    if (y >= p.H) return;
    const size_t plane = (size_t)p.H * p.W;
    const int nf = fold_count(p.W, p.R);
    if (p.W <= 2 * p.R) {   // narrow frame: several reflections, gather from global memory
        for (int j = lane; j < nf; j += 32) {
            const int x = fold_index(p.W, p.R, j);
            float v = 0.0f;
            for (int i = 0; i < p.K; ++i) {
                const int r = p.r[i];
                if (x >= r && x <= p.W - 1 - r) continue;
                v += adj1d_mirror(p.Y + plane * i + (size_t)y * p.W, 1, p.W, x, p.w + p.woff[i], r);
            }
            p.gimg[(size_t)y * p.W + x] += v;
        }
        return;
    }
    float* sl = edge[wq][0];   // Y_i(y, 0 .. r-1)
    float* sr = edge[wq][1];   // Y_i(y, W-r .. W-1)
    float v[(2 * DOG_MAX_RADIUS + 31) / 32];
#pragma unroll
    for (int k = 0; k < (2 * DOG_MAX_RADIUS + 31) / 32; ++k) v[k] = 0.0f;
    for (int i = 0; i < p.K; ++i) {
        const int r = p.r[i];
        const float* row = p.Y + plane * i + (size_t)y * p.W;
        __syncwarp();
        for (int n = lane; n < r; n += 32) {
            sl[n] = row[n];
            sr[n] = row[p.W - r + n];
        }
        __syncwarp();
        const float* w = p.w + p.woff[i];   // w[r + d] weighs offset d
#pragma unroll
        for (int k = 0; k < (2 * DOG_MAX_RADIUS + 31) / 32; ++k) {
            const int j = lane + 32 * k;
            if (j >= nf) break;
            const int x = fold_index(p.W, p.R, j);
            float acc = 0.0f;
            if (x < r) {   // reflected copy q = -1 - x: sum_{n=0}^{r-1-x} w[r + q - n] Y(n)
                for (int n = 0; n <= r - 1 - x; ++n) acc = __fmaf_rn(__ldg(w + r - 1 - x - n), sl[n], acc);
            } else if (x > p.W - 1 - r) {   // q = 2W - 1 - x: sum_{n=q-r}^{W-1} w[r + q - n] Y(n)
                const int q = 2 * p.W - 1 - x;
                for (int n = q - r; n <= p.W - 1; ++n) acc = __fmaf_rn(__ldg(w + r + q - n), sr[n - (p.W - r)], acc);
            }
            v[k] += acc;
        }
    }
#pragma unroll
    for (int k = 0; k < (2 * DOG_MAX_RADIUS + 31) / 32; ++k) {
        const int j = lane + 32 * k;
        if (j < nf) p.gimg[(size_t)y * p.W + fold_index(p.W, p.R, j)] += v[k];
    }
}

constexpr int ADJ_XR = 32;     // output rows per CTA of the row adjoint (4 warps x 8)

__host__ __device__ inline int adj_x_stride_y(int tpad_max) { return (32 + tpad_max + 8) | 1; }
__host__ __device__ inline int adj_x_stride_i(int R) { return (32 + 2 * R + 16) | 1; }
__host__ __device__ inline int adj_x_smem_floats(int tpad_max, int R, bool sig) {
    return ADJ_XR * (adj_x_stride_y(tpad_max) + (sig ? adj_x_stride_i(R) : 0)) + 2 * tpad_max;
}

// Row adjoint summed over levels into dloss/dI, and the kernel-shape part of
// dloss/dsigma_i = <Y_i, B_x' I> + <Yd_i, B_x I>.  A CTA covers 32 columns x 32
// rows; lane (rho, g) of warp q owns row 8q + rho, columns 8g .. 8g+7.
template <bool SIG>
__global__ void __launch_bounds__(128) adj_x_kernel(const __grid_constant__ AdjParams p, int tpad_max) {
    extern __shared__ float xsm[];
    __shared__ double red[4][MAX_LEVELS];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int rho = lane >> 2, g4 = lane & 3;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * ADJ_XR;
    const int row = 8 * q + rho;                 // 0 .. 31
    const int y = y0 + row;
    const int SY = adj_x_stride_y(tpad_max), SI = adj_x_stride_i(p.R);
    float* Yt = xsm;                              // ADJ_XR x SY: Y_i rows, columns x0 - r + c, zero outside
    float* It = Yt + ADJ_XR * SY;                 // ADJ_XR x SI: image rows, columns x0 - R + c, reflected
    float* ws = SIG ? It + ADJ_XR * SI : It;      // tpad_max (no image tile without SIG)
    float* wd = ws + tpad_max;                    // tpad_max
    const size_t plane = (size_t)p.H * p.W;
    const int R = p.R;
    // image rows y0 .. y0+31 (clamped), columns x0-R .. x0+R+47 (reflected);
    // thread t stages columns t, t + 128 of every row
    if (SIG) {
        const int c0 = threadIdx.x, c1 = threadIdx.x + 128;
        const int xr0 = refl_i(x0 - R + c0, p.W), xr1 = refl_i(x0 - R + c1, p.W);
        const bool ok0 = c0 < 32 + 2 * R + 16, ok1 = c1 < 32 + 2 * R + 16;
        for (int rr0 = 0; rr0 < ADJ_XR; rr0 += 8) {   // 16 loads in flight before the stores
            float v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float* src = p.img + (size_t)min(y0 + rr0 + u, p.H - 1) * p.pitch;
                v0[u] = ok0 ? __ldg(src + xr0) : 0.0f;
                v1[u] = ok1 ? __ldg(src + xr1) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (c0 < SI) It[(rr0 + u) * SI + c0] = v0[u];
                if (c1 < SI) It[(rr0 + u) * SI + c1] = v1[u];
            }
        }
    }
    float gsum[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) gsum[k] = 0.0f;
    for (int i = 0; i < p.K; ++i) {
        const int r = p.r[i], tpad = p.tpad[i], nb = tpad >> 3;
        const float* Yi = p.Y + plane * i;
        const float* Ydi = p.Yd + plane * i;
        __syncthreads();
        for (int t = threadIdx.x; t < tpad; t += blockDim.x) {
            ws[t] = p.w[p.woff[i] + t];
            wd[t] = p.dw[p.woff[i] + t];
        }
        const int wt = 32 + tpad + 8;
        // Y_i rows y0 .. y0+31, columns x0-r .. x0-r+wt-1 (zero outside the frame)
        const int xs = x0 - r;
        const int xa = xs >= 0 ? xs & ~3 : -((3 - xs) & ~3);   // xs rounded down to a multiple of 4
        const int off = xs - xa, n4 = (wt + off + 3) >> 2;     // float4 columns per row
        if ((p.W & 3) == 0 && xa >= 0 && xa + 4 * n4 <= p.W && y0 + ADJ_XR <= p.H) {
            // interior tile: 16-byte loads, thread (row phase, float4 column),
            // four rows' loads in flight
            const int rpp = 128 / n4, r0 = threadIdx.x / n4, c4 = threadIdx.x - r0 * n4;
            if (r0 < rpp) {
                const float4* src = reinterpret_cast<const float4*>(Yi + (size_t)y0 * p.W + xa) + c4;
                const int row4 = p.W >> 2;
                for (int rb = r0; rb < ADJ_XR; rb += 4 * rpp) {
                    float4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rr = min(rb + u * rpp, ADJ_XR - 1);
                        v[u] = __ldg(src + (size_t)rr * row4);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rr = rb + u * rpp;
                        if (rr < ADJ_XR) {
                            float* d = Yt + rr * SY + 4 * c4 - off;   // column 4 c4 + k - off of the tile
                            const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (4 * c4 + k - off >= 0 && 4 * c4 + k - off < wt) d[k] = e[k];
                        }
                    }
                }
            }
        } else {
            const int c0 = threadIdx.x, c1 = threadIdx.x + 128;
            const int xx0 = xs + c0, xx1 = xs + c1;
            const bool ok0 = c0 < wt && xx0 >= 0 && xx0 < p.W, ok1 = c1 < wt && xx1 >= 0 && xx1 < p.W;
            for (int rr0 = 0; rr0 < ADJ_XR; rr0 += 8) {   // 16 loads in flight before the stores
                float v0[8], v1[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int yy = y0 + rr0 + u;
                    const float* src = Yi + (size_t)yy * p.W;
                    v0[u] = (ok0 && yy < p.H) ? src[xx0] : 0.0f;
                    v1[u] = (ok1 && yy < p.H) ? src[xx1] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (c0 < wt) Yt[(rr0 + u) * SY + c0] = v0[u];
                    if (c1 < wt) Yt[(rr0 + u) * SY + c1] = v1[u];
                }
            }
        }
        __syncthreads();
        float z[8], hb[8], hd[8];
        corr8(Yt + row * SY + 8 * g4, 1, ws, nb, z);
        if (SIG) corr8x2(It + row * SI + (R - r) + 8 * g4, 1, ws, wd, nb, hb, hd);    // B_x I and B_x' I
        // this thread's 16 products in FP32 (one rounding each, as the inputs
        // are FP32), then the warp's sum in FP64 (the FP64 pipe is slow here)
        float dotf = 0.0f;
        if (y < p.H) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int x = x0 + 8 * g4 + k;
                if (x >= p.W) break;
                gsum[k] += z[k];
                if (SIG) {
                    const float yv = Yt[row * SY + r + 8 * g4 + k];   // Y_i(y, x)
                    dotf = __fmaf_rn(yv, hd[k], __fmaf_rn(Ydi[(size_t)y * p.W + x], hb[k], dotf));
                }
            }
        }
        if (SIG) {
            double dot = (double)dotf;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            if (lane == 0) red[q][i] = dot;
        }
    }
    if (y < p.H) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + 8 * g4 + k;
            if (x < p.W) p.gimg[(size_t)y * p.W + x] = gsum[k];
        }
    }
    if (!SIG) return;
    __syncthreads();
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < 4; ++w) s += red[w][i];
        if (s != 0.0) atomicAdd(&p.dw_acc[i], s);
    }
}

struct FinParams {
    const float* sig;
    int K, P, norm;
    double lref0, lrefP;
    const double* acc;   // dc (P), dt (P), dw (K)
    float* gsig;
};

__global__ void soft_finalize_kernel(const __grid_constant__ FinParams p) {
    const int i = threadIdx.x;
    if (i >= p.K) return;
    const double* dc = p.acc;
    const double* dt = p.acc + p.P;
    const double* dwt = p.acc + 2 * p.P;
    double g = dwt[i];
    const double si = (double)p.sig[i];
    if (p.norm == DOG_NORM_PAPER) {
        if (i < p.P) g += dc[i];
    } else {
        if (i < p.P) {
            const double d = (double)p.sig[i + 1] - si;
            g += dc[i] * (double)p.sig[i + 1] / (d * d);
        }
        if (i > 0) {
            const double d = si - (double)p.sig[i - 1];
            g -= dc[i - 1] * (double)p.sig[i - 1] / (d * d);
        }
    }
    if (i < p.P) g += dt[i] / (si * (p.lrefP - p.lref0));
    p.gsig[i] += (float)g;
}

// dloss/dL planes from a recorded list of maxima: A_l += c_l G_v and
// A_{l+1} -= c_l G_v for a maximum v in plane l, G_v = gk_l q_v with
// gk_l = sum_b gH_b kappa_b(t_l); dloss/dc_l += gk_l qe_v, dloss/dt_l +=
// s_v sum_b gH_b dkappa_b(t_l).  A must be zero beforehand.
struct ScatterParams {
    const dog_soft_max* rec;
    const int* count;
    int cap;
    const float* gH;
    const float* kappa;
    const float* dkappa;
    const float* c;
    int P, nbins, H, W;
    float* A;
    double* dc_acc;
    double* dt_acc;
    int* status;
};

__global__ void __launch_bounds__(256) soft_scatter_kernel(const __grid_constant__ ScatterParams p) {
    __shared__ float gk[MAX_LEVELS], gdk[MAX_LEVELS], cl[MAX_LEVELS], dc[MAX_LEVELS], dt[MAX_LEVELS];
    for (int l = threadIdx.x; l < p.P; l += blockDim.x) {
        float a = 0.0f, b = 0.0f;
        for (int k = 0; k < p.nbins; ++k) {
            a += p.gH[k] * p.kappa[l * p.nbins + k];
            b += p.gH[k] * p.dkappa[l * p.nbins + k];
        }
        gk[l] = a;
        gdk[l] = b;
        cl[l] = p.c[l];
        dc[l] = 0.0f;
        dt[l] = 0.0f;
    }
    __syncthreads();
    const int n = *p.count;
    if (n > p.cap && blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
    const int m = min(n, p.cap);
    const size_t plane = (size_t)p.H * p.W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const dog_soft_max v = p.rec[i];
        const int l = v.level;
        if (v.x < 0 || v.x >= p.W || v.y < 0 || v.y >= p.H || l < 0 || l >= p.P) {   // not this frame's record
            atomicCAS(p.status, 0, (int)DOG_ERR_INVALID);
            continue;
        }
        const float G = gk[l] * v.q;
        const size_t pix = (size_t)v.y * p.W + v.x;
        atomicAdd(&p.A[plane * l + pix], cl[l] * G);
        atomicAdd(&p.A[plane * (l + 1) + pix], -cl[l] * G);
        atomicAdd(&dc[l], gk[l] * v.qe);
        atomicAdd(&dt[l], v.s * gdk[l]);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < p.P; l += blockDim.x) {
        if (dc[l] != 0.0f) atomicAdd(&p.dc_acc[l], (double)dc[l]);
        if (dt[l] != 0.0f) atomicAdd(&p.dt_acc[l], (double)dt[l]);
    }
}

// Kernel-shape part of dloss/dsigma from a recorded list of maxima.  A_m is
// nonzero only at the maxima's pixels (A_l += c_l G_v, A_{l+1} -= c_l G_v for a
// maximum v in plane l), so
//   sum_x A_m(x) dL_m/dsigma_m(x),  dL_m/dsigma_m = B_y' B_x I + B_y B_x' I,
// is evaluated at those pixels only: for a maximum v in plane l, the sums of
// (w'_j w_t + w_j w'_t) I(y + j, x + t) over |j|, |t| <= r_m of the reflected
// image for m = l and m = l + 1 at once.  Windows at most 31 wide take one
// warp (lanes on columns, several rows per pass); wider ones (the few maxima
// of the coarse planes) are queued for a second kernel that gives each one a
// whole CTA, so that no warp runs a long serial window.  Per-CTA sums in FP64
// shared memory, one global atomic per level.
struct SigmaParams {
    const dog_soft_max* rec;
    const int* count;
    int cap;
    const float* gH;
    const float* kappa;
    const float* c;
    const float* w;
    const float* dw;
    const float* img;
    int pitch;
    int P, nbins, H, W;
    int r[MAX_LEVELS];
    int woff[MAX_LEVELS];
    int* big;          // queue of wide-window maxima (record indices)
    int* big_count;
    int big_cap;
    double* dw_acc;
};

constexpr int SIGMA_WIDE_R = 16;   // windows of radius >= this go to the CTA kernel

// Partial window sums of maximum v for planes l (pa) and l + 1 (pb): columns
// t0, t0 + dt_step, ... and rows j0, j0 + j_step, ... of the (2 R2 + 1)^2
// window, four rows' loads in flight.
__device__ __forceinline__ void sigma_sums(const SigmaParams& p, const dog_soft_max& v, int t0, int t_step, int j0,
                                           int j_step, float& pa, float& pb) {
    const int l = v.level;
    const int ra = p.r[l], rb = p.r[l + 1], R2 = max(ra, rb), n2 = 2 * R2 + 1;
    const float* wa = p.w + p.woff[l];
    const float* wda = p.dw + p.woff[l];
    const float* wb = p.w + p.woff[l + 1];
    const float* wdb = p.dw + p.woff[l + 1];
    for (int t = t0; t < n2; t += t_step) {
        const int dt = t - R2;
        // this lane's column weights (zero outside a plane's window)
        const bool ia = dt >= -ra && dt <= ra, ib = dt >= -rb && dt <= rb;
        const float wat = ia ? __ldg(wa + dt + ra) : 0.0f, wdat = ia ? __ldg(wda + dt + ra) : 0.0f;
        const float wbt = ib ? __ldg(wb + dt + rb) : 0.0f, wdbt = ib ? __ldg(wdb + dt + rb) : 0.0f;
        const float* col = p.img + refl_i(v.x + dt, p.W);
        for (int jb = j0; jb < n2; jb += 4 * j_step) {
            float px[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = min(jb + u * j_step, n2 - 1);
                px[u] = __ldg(col + (size_t)refl_i(v.y + j - R2, p.H) * p.pitch);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jb + u * j_step, dj = j - R2;
                if (j < n2) {
                    if (dj >= -ra && dj <= ra)
                        pa = __fmaf_rn(__fmaf_rn(__ldg(wda + dj + ra), wat, __ldg(wa + dj + ra) * wdat), px[u], pa);
                    if (dj >= -rb && dj <= rb)
                        pb = __fmaf_rn(__fmaf_rn(__ldg(wdb + dj + rb), wbt, __ldg(wb + dj + rb) * wdbt), px[u], pb);
                }
            }
        }
    }
}

__device__ __forceinline__ void sigma_prologue(const SigmaParams& p, float* gk, float* cl, double* acc) {
    for (int l = threadIdx.x; l < MAX_LEVELS; l += blockDim.x) {
        float a = 0.0f;
        if (l < p.P)
            for (int k = 0; k < p.nbins; ++k) a += p.gH[k] * p.kappa[l * p.nbins + k];
        gk[l] = a;
        cl[l] = l < p.P ? p.c[l] : 0.0f;
        acc[l] = 0.0;
    }
    __syncthreads();
}

__device__ __forceinline__ void sigma_epilogue(const SigmaParams& p, const double* acc) {
    __syncthreads();
    for (int l = threadIdx.x; l < MAX_LEVELS; l += blockDim.x)
        if (acc[l] != 0.0) atomicAdd(&p.dw_acc[l], acc[l]);
}

__device__ __forceinline__ bool sigma_valid(const SigmaParams& p, const dog_soft_max& v) {
    return v.x >= 0 && v.x < p.W && v.y >= 0 && v.y < p.H && v.level >= 0 && v.level < p.P;   // else flagged by the scatter
}

__global__ void __launch_bounds__(256) soft_sigma_kernel(const __grid_constant__ SigmaParams p) {
    __shared__ float gk[MAX_LEVELS], cl[MAX_LEVELS];
    __shared__ double acc[MAX_LEVELS];
    sigma_prologue(p, gk, cl, acc);
    const int lane = threadIdx.x & 31;
    const int nmax = min(*p.count, p.cap);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < nmax; task += nwarps) {
        const dog_soft_max v = p.rec[task];
        if (!sigma_valid(p, v)) continue;
        const int l = v.level;
        const int R2 = max(p.r[l], p.r[l + 1]), n2 = 2 * R2 + 1;
        float pa = 0.0f, pb = 0.0f;
        if (R2 >= SIGMA_WIDE_R) {
            int k = 0;
            if (lane == 0) k = atomicAdd(p.big_count, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < p.big_cap) {   // queued for the CTA kernel
                if (lane == 0) p.big[k] = task;
                continue;
            }
            sigma_sums(p, v, lane, 32, 0, 1, pa, pb);   // queue full: this warp takes it
        } else {
            const int rpi = 32 / n2, js = lane / n2;   // rows per pass, this lane's row phase
            if (js < rpi) sigma_sums(p, v, lane - js * n2, n2, js, rpi, pa, pb);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pa += __shfl_xor_sync(0xffffffffu, pa, o);
            pb += __shfl_xor_sync(0xffffffffu, pb, o);
        }
        if (lane == 0) {
            const double G = (double)(cl[l] * (gk[l] * v.q));
            atomicAdd(&acc[l], G * (double)pa);
            atomicAdd(&acc[l + 1], -G * (double)pb);
        }
    }
    sigma_epilogue(p, acc);
}

// The queued wide windows: one CTA per maximum, warp w on window rows
// w, w + 8, ..., lanes on columns.
__global__ void __launch_bounds__(256) soft_sigma_wide_kernel(const __grid_constant__ SigmaParams p) {
    __shared__ float gk[MAX_LEVELS], cl[MAX_LEVELS];
    __shared__ double acc[MAX_LEVELS];
    sigma_prologue(p, gk, cl, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbig = min(*p.big_count, p.big_cap);
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const dog_soft_max v = p.rec[p.big[q]];
        const int l = v.level;
        float pa = 0.0f, pb = 0.0f;
        sigma_sums(p, v, lane, 32, warp, 8, pa, pb);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pa += __shfl_xor_sync(0xffffffffu, pa, o);
            pb += __shfl_xor_sync(0xffffffffu, pb, o);
        }
        if (lane == 0) {
            const double G = (double)(cl[l] * (gk[l] * v.q));
            atomicAdd(&acc[l], G * (double)pa);
            atomicAdd(&acc[l + 1], -G * (double)pb);
        }
    }
    sigma_epilogue(p, acc);
}

static int adjoint_tail(dog_handle* h, SoftWS* ws, const SoftPrep& q, const float* img, int H, int W, int pitch,
                        const float* sig, float* gimg, float* gsig, bool dense_sigma, cudaStream_t s);

int soft_backward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig,
                  const float* gH, float* gimg, float* gsig, cudaStream_t s) {
    SoftWS* ws = nullptr;
    int st = soft_ws(h, H, W, &ws);
    if (st != DOG_OK) return st;
    SoftPrep q = prep_params(h, ws, sig);
    soft_prep_kernel<<<1, PREP_THREADS, 0, s>>>(q);
    SOFT_CUDA(cudaGetLastError());
    const FusedParams& b = handle_base(h);
    const int K = b.K, P = b.P;
    SOFT_CUDA(cudaMemsetAsync(ws->counts, 0, sizeof(int) * 4, s));
    SOFT_CUDA(cudaMemsetAsync(ws->acc, 0, sizeof(double) * (2 * P + K), s));
    FusedParams p = soft_fused(h, ws, img, H, W, pitch, MODE_BWD);
    p.gH = gH;
    p.A = ws->A;
    p.dc_acc = ws->acc;
    p.dt_acc = ws->acc + P;
    SOFT_CUDA(timed_fused(h, p, p.n_strips * p.n_bands, s));
    return adjoint_tail(h, ws, q, img, H, W, pitch, sig, gimg, gsig, true, s);
}

int soft_backward_rec(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig,
                      const dog_soft_max* rec, const int* rec_count, int rec_cap, const float* gH, float* gimg,
                      float* gsig, cudaStream_t s) {
    SoftWS* ws = nullptr;
    int st = soft_ws(h, H, W, &ws);
    if (st != DOG_OK) return st;
    SoftPrep q = prep_params(h, ws, sig);
    soft_prep_kernel<<<1, PREP_THREADS, 0, s>>>(q);
    SOFT_CUDA(cudaGetLastError());
    const FusedParams& b = handle_base(h);
    const int K = b.K, P = b.P;
    SOFT_CUDA(cudaMemsetAsync(ws->acc, 0, sizeof(double) * (2 * P + K), s));
    SOFT_CUDA(cudaMemsetAsync(ws->A, 0, sizeof(float) * (size_t)K * H * W, s));
    ScatterParams c{};
    c.rec = rec;
    c.count = rec_count;
    c.cap = rec_cap;
    c.gH = gH;
    c.kappa = ws->kappa;
    c.dkappa = ws->dkappa;
    c.c = ws->c;
    c.P = P;
    c.nbins = handle_cfg(h).nbins;
    c.H = H;
    c.W = W;
    c.A = ws->A;
    c.dc_acc = ws->acc;
    c.dt_acc = ws->acc + P;
    c.status = handle_status(h);
    const int grid = std::max(1, std::min((rec_cap + 255) / 256, 152 * 8));
    soft_scatter_kernel<<<grid, 256, 0, s>>>(c);
    SOFT_CUDA(cudaGetLastError());
    SigmaParams g{};
    g.rec = rec;
    g.count = rec_count;
    g.cap = rec_cap;
    g.gH = gH;
    g.kappa = ws->kappa;
    g.c = ws->c;
    g.w = ws->w;
    g.dw = ws->dw;
    g.img = img;
    g.pitch = pitch;
    g.P = P;
    g.nbins = handle_cfg(h).nbins;
    g.H = H;
    g.W = W;
    for (int i = 0; i < K; ++i) {
        g.r[i] = b.lv[i].r;
        g.woff[i] = b.lv[i].woff;
    }
    g.dw_acc = ws->acc + 2 * P;
    g.big = ws->big;
    g.big_count = ws->big_count;
    g.big_cap = ws->big_cap;
    SOFT_CUDA(cudaMemsetAsync(ws->big_count, 0, sizeof(int), s));
    soft_sigma_kernel<<<152 * 4, 256, 0, s>>>(g);
    SOFT_CUDA(cudaGetLastError());
    soft_sigma_wide_kernel<<<152 * 4, 256, 0, s>>>(g);
    SOFT_CUDA(cudaGetLastError());
    return adjoint_tail(h, ws, q, img, H, W, pitch, sig, gimg, gsig, false, s);
}

// The adjoint blurs of the dloss/dL planes in ws->A, then the sigma gradient.
static int adjoint_tail(dog_handle* h, SoftWS* ws, const SoftPrep& q, const float* img, int H, int W, int pitch,
                        const float* sig, float* gimg, float* gsig, bool dense_sigma, cudaStream_t s) {
    const FusedParams& b = handle_base(h);
    const int K = b.K, P = b.P;
    AdjParams a{};
    a.A = ws->A;
    a.Y = ws->Y;
    a.Yd = ws->Yd;
    a.img = img;
    a.pitch = pitch;
    a.gimg = gimg;
    a.H = H;
    a.W = W;
    a.K = K;
    a.w = ws->w;
    a.dw = ws->dw;
    int tpad_max = 8;
    for (int i = 0; i < K; ++i) {
        a.r[i] = b.lv[i].r;
        a.tpad[i] = b.lv[i].tpad;
        a.woff[i] = b.lv[i].woff;
        tpad_max = std::max(tpad_max, b.lv[i].tpad);
    }
    a.R = b.R;
    a.dw_acc = ws->acc + 2 * P;
    dim3 gy((W + 31) / 32, (H + ADJ_TM - 1) / ADJ_TM, K);
    dim3 gyf((W + 127) / 128, fold_count(H, b.R), K);
    dim3 gx((W + 31) / 32, (H + ADJ_XR - 1) / ADJ_XR);
    if (dense_sigma) {
        adj_y_kernel<true><<<gy, 256, sizeof(float) * adj_y_smem_floats(tpad_max), s>>>(a);
        adj_y_fold_kernel<true><<<gyf, 128, 0, s>>>(a);
        adj_x_kernel<true><<<gx, 128, sizeof(float) * adj_x_smem_floats(tpad_max, b.R, true), s>>>(a, tpad_max);
    } else {
        adj_y_kernel<false><<<gy, 256, sizeof(float) * adj_y_smem_floats(tpad_max), s>>>(a);
        adj_y_fold_kernel<false><<<gyf, 128, 0, s>>>(a);
        adj_x_kernel<false><<<gx, 128, sizeof(float) * adj_x_smem_floats(tpad_max, b.R, false), s>>>(a, tpad_max);
    }
    SOFT_CUDA(cudaGetLastError());
    adj_x_fold_kernel<<<(H + FOLD_ROWS - 1) / FOLD_ROWS, 32 * FOLD_ROWS, 0, s>>>(a);
    SOFT_CUDA(cudaGetLastError());
    FinParams f{};
    f.sig = sig;
    f.K = K;
    f.P = P;
    f.norm = handle_cfg(h).norm;
    f.lref0 = q.lref0;
    f.lrefP = q.lrefP;
    f.acc = ws->acc;
    f.gsig = gsig;
    soft_finalize_kernel<<<1, 64, 0, s>>>(f);
    SOFT_CUDA(cudaGetLastError());
    return DOG_OK;
}

}  // namespace dogk
