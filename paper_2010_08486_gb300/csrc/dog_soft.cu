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
// The forward L_i are recomputed by the fused kernel (MODE_BWD), which also
// writes A densely; the adjoint blurs gather through the reflect fold-back.
#include <cuda_runtime.h>

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
};

void soft_free(dog_handle* h) {
    SoftWS* ws = static_cast<SoftWS*>(handle_soft_ws(h));
    if (!ws) return;
    void* ptrs[] = {ws->w, ws->dw, ws->c, ws->kappa, ws->dkappa, ws->pend, ws->counts, ws->A, ws->Y, ws->Yd, ws->acc};
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
};

__global__ void __launch_bounds__(256) soft_prep_kernel(const __grid_constant__ SoftPrep p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < p.K; i += 8) {
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
    p.n_strips = (W + TX - 1) / TX;
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

static ResolveParams soft_resolve(dog_handle* h, const FusedParams& f) {
    ResolveParams r{};
    r.pend = f.pend;
    r.pend_count = f.pend_count;
    r.pend_cap = f.pend_cap;
    r.img = f.img;
    r.dtype = f.dtype;
    r.H = f.H;
    r.W = f.W;
    r.pitch = f.pitch;
    r.K = f.K;
    r.P = f.P;
    r.w = f.w;
    r.c = f.c;
    for (int i = 0; i < f.K; ++i) {
        r.woff[i] = f.lv[i].woff;
        r.r[i] = f.lv[i].r;
    }
    r.mode = f.mode;
    r.kappa = f.kappa;
    r.dkappa = f.dkappa;
    r.gH = f.gH;
    r.nbins = f.nbins;
    r.thr = f.thr;
    r.inv_T = f.inv_T;
    r.soft_out = f.soft_out;
    r.A = f.A;
    r.dc_acc = f.dc_acc;
    r.dt_acc = f.dt_acc;
    r.status = handle_status(h);
    (void)h;
    return r;
}

#define SOFT_CUDA(x)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA; \
    } while (0)

int soft_forward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig, float* out,
                 cudaStream_t s) {
    SoftWS* ws = nullptr;
    int st = soft_ws(h, H, W, &ws);
    if (st != DOG_OK) return st;
    SoftPrep q = prep_params(h, ws, sig);
    soft_prep_kernel<<<1, 256, 0, s>>>(q);
    SOFT_CUDA(cudaGetLastError());
    SOFT_CUDA(cudaMemsetAsync(ws->counts, 0, sizeof(int) * 4, s));
    FusedParams p = soft_fused(h, ws, img, H, W, pitch, MODE_SOFT);
    p.soft_out = out;
    SOFT_CUDA(timed_fused(h, p, p.n_strips * p.n_bands, s));
    SOFT_CUDA(launch_resolve(soft_resolve(h, p), std::min(ws->pend_cap, 152 * 64), s));
    return DOG_OK;
}

// ---------------------------------------------------------------------------
// 1-D adjoint of a reflect-boundary correlation with the symmetric full kernel
// w[0..2r] (w[r + d] weighs offset d), evaluated at index m of a line of length N with stride `st`:
// sum over the preimages q of m under the reflection that lie within r of the
// line, of sum_n w[|q-n|] a[n].
__device__ __forceinline__ float adj1d(const float* __restrict__ a, size_t st, int N, int m,
                                       const float* __restrict__ w, int r) {
    float acc = 0.0f;
    const int per = 2 * N;
    const int fam[2] = {m, per - 1 - m};
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        int q = fam[f];
        // first q of this family >= -r
        const int k = (-r - q) > 0 ? ((-r - q) + per - 1) / per : -((q + r) / per);
        for (q = q + k * per; q <= N - 1 + r; q += per) {
            const int nlo = max(0, q - r), nhi = min(N - 1, q + r);
            for (int n = nlo; n <= nhi; ++n) acc = __fmaf_rn(__ldg(w + r + (q - n)), __ldg(a + (size_t)n * st), acc);
        }
    }
    return acc;
}

__device__ __forceinline__ int refl_i(int i, int n) {
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
    int H, W, K;
    const float* w;
    const float* dw;
    int r[MAX_LEVELS];
    int woff[MAX_LEVELS];
    double* dw_acc;
};

// Column adjoint of every level: Y_i = B_y^T A_i (kernel w_i), Yd_i (kernel dw_i).
__global__ void __launch_bounds__(256) adj_y_kernel(const __grid_constant__ AdjParams p) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int i = blockIdx.z;
    if (x >= p.W || y >= p.H) return;
    const size_t plane = (size_t)p.H * p.W;
    const float* a = p.A + plane * i + x;
    const int r = p.r[i];
    p.Y[plane * i + (size_t)y * p.W + x] = adj1d(a, p.W, p.H, y, p.w + p.woff[i], r);
    p.Yd[plane * i + (size_t)y * p.W + x] = adj1d(a, p.W, p.H, y, p.dw + p.woff[i], r);
}

// Row adjoint summed over levels into dloss/dI, and the kernel-shape part of
// dloss/dsigma_i = <Y_i, B_x' I> + <Yd_i, B_x I>.
__global__ void __launch_bounds__(256) adj_x_kernel(const __grid_constant__ AdjParams p) {
    __shared__ double red[8][MAX_LEVELS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int y = blockIdx.y * 8 + warp;
    const bool ok = x < p.W && y < p.H;
    const size_t plane = (size_t)p.H * p.W;
    float g = 0.0f;
    for (int i = 0; i < p.K; ++i) {
        double dot = 0.0;
        if (ok) {
            const int r = p.r[i];
            const float* w = p.w + p.woff[i];
            const float* dw = p.dw + p.woff[i];
            g += adj1d(p.Y + plane * i + (size_t)y * p.W, 1, p.W, x, w, r);
            float hb = 0.0f, hd = 0.0f;
            const float* row = p.img + (size_t)y * p.pitch;
            for (int k = -r; k <= r; ++k) {
                const float v = __ldg(row + refl_i(x + k, p.W));
                hb = __fmaf_rn(__ldg(w + r + k), v, hb);
                hd = __fmaf_rn(__ldg(dw + r + k), v, hd);
            }
            const size_t o = plane * i + (size_t)y * p.W + x;
            dot = (double)p.Y[o] * (double)hd + (double)p.Yd[o] * (double)hb;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) red[warp][i] = dot;
    }
    if (ok) p.gimg[(size_t)y * p.W + x] = g;
    __syncthreads();
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += red[q][i];
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

int soft_backward(dog_handle* h, const float* img, int H, int W, int pitch, const float* sig,
                  const float* gH, float* gimg, float* gsig, cudaStream_t s) {
    SoftWS* ws = nullptr;
    int st = soft_ws(h, H, W, &ws);
    if (st != DOG_OK) return st;
    SoftPrep q = prep_params(h, ws, sig);
    soft_prep_kernel<<<1, 256, 0, s>>>(q);
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
    SOFT_CUDA(launch_resolve(soft_resolve(h, p), std::min(ws->pend_cap, 152 * 64), s));
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
    for (int i = 0; i < K; ++i) {
        a.r[i] = b.lv[i].r;
        a.woff[i] = b.lv[i].woff;
    }
    a.dw_acc = ws->acc + 2 * P;
    dim3 gy((W + 31) / 32, (H + 7) / 8, K);
    adj_y_kernel<<<gy, 256, 0, s>>>(a);
    SOFT_CUDA(cudaGetLastError());
    dim3 gx((W + 31) / 32, (H + 7) / 8);
    adj_x_kernel<<<gx, 256, 0, s>>>(a);
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
