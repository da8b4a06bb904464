// FFT-convolution backend of the scale space (Sec. 4.1 names FFT convolution
// as the alternative to direct convolution; Sec. 5 compares the two).
//
// Per frame: the frame is reflect-padded by R (the largest radius, with the
// same half-sample fold as the direct path) into a grid of Hp x Wp cells
// (2-3-5-7-smooth sizes, Hp >= max_h + 2R, Wp >= max_w + 2R, zeros beyond);
// one real-to-complex FFT; for every level the spectrum is multiplied by the
// level's kernel spectrum, which is real and separable (the sampled Gaussian
// is even): G_i(ky, kx) = g_i(ky) g_i(kx), g(k) = w_0 + 2 sum_t w_t cos(2 pi k
// t / N), computed in double on the host; one batched complex-to-real inverse
// FFT gives every L_i on the grid, where the frame's pixel (y, x) sits at
// (y + R, x + R) and no circular wrap reaches it (the kernels span at most R).
// A stencil kernel then forms D_l = c_l (L_l - L_{l+1}) and applies the same
// 3x3x3 test and strict threshold as the direct path, compacting candidates
// with one atomic each.  The FFTs run in single precision (cuFFT); the values
// differ from the direct sums by the transforms' rounding.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <vector>

#include "dog_internal.cuh"
#include "dog_device.cuh"

namespace dogk {

struct FftWS {
    int Hp = 0, Wp = 0, K = 0, R = 0;
    int last_h = 0, last_w = 0;   // frame size of the last padding (grid cells past it are zero)
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    float* pad = nullptr;         // Hp x Wp
    cufftComplex* spec = nullptr; // Hp x (Wp/2+1)
    cufftComplex* specs = nullptr;  // K x Hp x (Wp/2+1)
    float* planes = nullptr;      // K x Hp x Wp
    float* gx = nullptr;          // K x (Wp/2+1) kernel spectra along x (divided by Hp Wp)
    float* gy = nullptr;          // K x Hp kernel spectra along y
};

// smallest n >= m whose prime factors are 2, 3, 5 and 7
int fft_size(int m) {
    for (int n = m > 1 ? m : 1;; ++n) {
        int v = n;
        for (int p : {2, 3, 5, 7})
            while (v % p == 0) v /= p;
        if (v == 1) return n;
    }
}

void fft_free(FftWS* f) {
    if (!f) return;
    if (f->have_fwd) cufftDestroy(f->fwd);
    if (f->have_inv) cufftDestroy(f->inv);
    void* ptrs[] = {f->pad, f->spec, f->specs, f->planes, f->gx, f->gy};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

// Workspace and plans for frames up to max_h x max_w; kernel spectra of the
// handle's ladder (w: K kernels of 2 r_i + 1 taps, tap t weighing offset t - r).
int fft_create(FftWS** out, int max_h, int max_w, int K, int R, const std::vector<std::vector<double>>& w) {
    FftWS* f = new (std::nothrow) FftWS();
    if (!f) return DOG_ERR_NOMEM;
    f->Hp = fft_size(max_h + 2 * R);
    f->Wp = fft_size(max_w + 2 * R);
    f->K = K;
    f->R = R;
    const int Wc = f->Wp / 2 + 1;
    const size_t n_pad = (size_t)f->Hp * f->Wp, n_spec = (size_t)f->Hp * Wc;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(cudaMalloc(&f->pad, sizeof(float) * n_pad));
    ok(cudaMalloc(&f->spec, sizeof(cufftComplex) * n_spec));
    ok(cudaMalloc(&f->specs, sizeof(cufftComplex) * n_spec * K));
    ok(cudaMalloc(&f->planes, sizeof(float) * n_pad * K));
    ok(cudaMalloc(&f->gx, sizeof(float) * (size_t)K * Wc));
    ok(cudaMalloc(&f->gy, sizeof(float) * (size_t)K * f->Hp));
    if (e == cudaSuccess) ok(cudaMemset(f->pad, 0, sizeof(float) * n_pad));
    if (e != cudaSuccess) {
        fft_free(f);
        return e == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA;
    }
    // kernel spectra, double on the host, rounded to float; 1 / (Hp Wp) (the
    // inverse transform's scale) folded into gx
    std::vector<float> hx((size_t)K * Wc), hy((size_t)K * f->Hp);
    const double two_pi = 2.0 * M_PI, scale = 1.0 / ((double)f->Hp * (double)f->Wp);
    for (int i = 0; i < K; ++i) {
        const int r = ((int)w[i].size() - 1) / 2;
        for (int k = 0; k < Wc; ++k) {
            double g = w[i][r];
            for (int t = 1; t <= r; ++t) g += 2.0 * w[i][r + t] * std::cos(two_pi * (double)k * t / f->Wp);
            hx[(size_t)i * Wc + k] = (float)(g * scale);
        }
        for (int k = 0; k < f->Hp; ++k) {
            double g = w[i][r];
            for (int t = 1; t <= r; ++t) g += 2.0 * w[i][r + t] * std::cos(two_pi * (double)k * t / f->Hp);
            hy[(size_t)i * f->Hp + k] = (float)g;
        }
    }
    ok(cudaMemcpy(f->gx, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice));
    ok(cudaMemcpy(f->gy, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice));
    if (e == cudaSuccess) {
        if (cufftPlan2d(&f->fwd, f->Hp, f->Wp, CUFFT_R2C) != CUFFT_SUCCESS) e = cudaErrorUnknown;
        else f->have_fwd = true;
    }
    if (e == cudaSuccess) {
        int n[2] = {f->Hp, f->Wp};
        if (cufftPlanMany(&f->inv, 2, n, nullptr, 1, (int)n_spec, nullptr, 1, (int)n_pad, CUFFT_C2R, K) !=
            CUFFT_SUCCESS)
            e = cudaErrorUnknown;
        else
            f->have_inv = true;
    }
    if (e != cudaSuccess) {
        fft_free(f);
        return e == cudaErrorMemoryAllocation ? DOG_ERR_NOMEM : DOG_ERR_CUDA;
    }
    *out = f;
    return DOG_OK;
}

// Reflect-padded frame on the grid: cell (Y, X) for Y < H + 2R, X < W + 2R
// holds pixel (refl(Y - R), refl(X - R)); the rest of the grid stays zero.
__global__ void fft_pad_kernel(const void* img, int dtype, int H, int W, int pitch, const int* lohi, int R,
                               float* pad, int Wp) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= W + 2 * R) return;
    const int lo = dtype == DTYPE_U16_STRETCH ? lohi[0] : 0, hi = dtype == DTYPE_U16_STRETCH ? lohi[1] : 0;
    const float rcp = stretch_rcp(lo, hi);
    const int x = refl(X - R, W);
    for (int Y = blockIdx.y; Y < H + 2 * R; Y += gridDim.y)
        pad[(size_t)Y * Wp + X] = raw_to_px(load_raw(img, dtype, pitch, refl(Y - R, H), x), dtype, lo, hi, rcp);
}

// spectra of all levels: specs[i] = spec * gy[i][ky] * gx[i][kx]
__global__ void fft_levels_kernel(const cufftComplex* __restrict__ spec, const float* __restrict__ gx,
                                  const float* __restrict__ gy, int K, int Hp, int Wc, cufftComplex* specs) {
    const int kx = blockIdx.x * blockDim.x + threadIdx.x;
    if (kx >= Wc) return;
    const size_t n_spec = (size_t)Hp * Wc;
    for (int ky = blockIdx.y; ky < Hp; ky += gridDim.y) {
        const size_t o = (size_t)ky * Wc + kx;
        const cufftComplex s = spec[o];
        for (int i = 0; i < K; ++i) {
            const float g = __fmul_rn(gy[(size_t)i * Hp + ky], gx[(size_t)i * Wc + kx]);
            specs[(size_t)i * n_spec + o] = make_float2(__fmul_rn(s.x, g), __fmul_rn(s.y, g));
        }
    }
}

// DoG, 3x3x3 maximum and threshold from the level planes; one thread per
// pixel walks the planes with a window of three 3x3 neighbourhoods.
// Neighbours outside the frame or the ladder do not count (-inf); ties keep
// the voxel (it equals its maximum filter); strict threshold D > thr.
// mode MODE_CANDIDATES: compaction into blobs; MODE_DUMP: writes D.
__global__ void __launch_bounds__(256) fft_test_kernel(const float* __restrict__ planes, int Hp, int Wp, int R,
                                                       int H, int W, int P, const float* __restrict__ c, float thr,
                                                       int mode, dog_blob* blobs, int cap, int* count, float* dump,
                                                       int* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t plane = (size_t)Hp * Wp;
    const float NEG = -INFINITY;
    float Dw[3][9];   // D of planes l-1, l, l+1 around (y, x), row-major 3x3
    auto load = [&](int l, float (&d)[9]) {
        const float* a = planes + (size_t)l * plane;
        const float* b = a + plane;
        const float cl = c[l];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int yy = y + q / 3 - 1, xx = x + q % 3 - 1;
            const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t o = (size_t)(yy + R) * Wp + (xx + R);
            d[q] = in ? dog_value(cl, a[o], b[o]) : NEG;
        }
    };
#pragma unroll
    for (int q = 0; q < 9; ++q) Dw[0][q] = NEG;
    load(0, Dw[1]);
    for (int l = 0; l < P; ++l) {
        if (l + 1 < P) load(l + 1, Dw[2]);
        else
#pragma unroll
            for (int q = 0; q < 9; ++q) Dw[2][q] = NEG;
        const float d = Dw[1][4];
        if (mode == MODE_DUMP) {
            dump[((size_t)l * H + y) * W + x] = d;
        } else if (d > thr) {
            float m = NEG;
#pragma unroll
            for (int q = 0; q < 9; ++q) m = fmaxf(m, fmaxf(Dw[0][q], Dw[2][q]));
#pragma unroll
            for (int q = 0; q < 9; ++q)
                if (q != 4) m = fmaxf(m, Dw[1][q]);
            if (d >= m) {
                const int idx = atomicAdd(count, 1);
                if (idx < cap) {
                    dog_blob b;
                    b.x = x; b.y = y; b.level = l; b.sigma = c[P + l]; b.response = d;
                    blobs[idx] = b;
                } else {
                    atomicCAS(status, 0, (int)DOG_ERR_CAPACITY);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            Dw[0][q] = Dw[1][q];
            Dw[1][q] = Dw[2][q];
        }
    }
}

// The scale space of one frame on the FFT grid (planes), then the test.
int fft_run(FftWS* f, const void* img, int dtype, int H, int W, int pitch, const int* lohi, int P,
            const float* c, float thr, int mode, dog_blob* blobs, int cap, int* count, float* dump, int* status,
            cudaStream_t s) {
    if (H + 2 * f->R > f->Hp || W + 2 * f->R > f->Wp) return DOG_ERR_INVALID;
    const int Wc = f->Wp / 2 + 1;
    if ((H < f->last_h || W < f->last_w) &&   // cells a larger frame padded: back to zero
        cudaMemsetAsync(f->pad, 0, sizeof(float) * (size_t)f->Hp * f->Wp, s) != cudaSuccess)
        return DOG_ERR_CUDA;
    f->last_h = H;
    f->last_w = W;
    const int gy_pad = H + 2 * f->R < 65535 ? H + 2 * f->R : 65535;
    fft_pad_kernel<<<dim3((W + 2 * f->R + 255) / 256, gy_pad), 256, 0, s>>>(img, dtype, H, W, pitch, lohi, f->R,
                                                                           f->pad, f->Wp);
    if (cudaGetLastError() != cudaSuccess) return DOG_ERR_CUDA;
    if (cufftSetStream(f->fwd, s) != CUFFT_SUCCESS || cufftSetStream(f->inv, s) != CUFFT_SUCCESS) return DOG_ERR_CUDA;
    if (cufftExecR2C(f->fwd, f->pad, f->spec) != CUFFT_SUCCESS) return DOG_ERR_CUDA;
    fft_levels_kernel<<<dim3((Wc + 255) / 256, f->Hp < 65535 ? f->Hp : 65535), 256, 0, s>>>(f->spec, f->gx, f->gy,
                                                                                         f->K, f->Hp, Wc, f->specs);
    if (cudaGetLastError() != cudaSuccess) return DOG_ERR_CUDA;
    if (cufftExecC2R(f->inv, f->specs, f->planes) != CUFFT_SUCCESS) return DOG_ERR_CUDA;
    if (mode == MODE_CANDIDATES && cudaMemsetAsync(count, 0, sizeof(int), s) != cudaSuccess) return DOG_ERR_CUDA;
    fft_test_kernel<<<dim3((W + 255) / 256, H), 256, 0, s>>>(f->planes, f->Hp, f->Wp, f->R, H, W, P, c, thr, mode,
                                                             blobs, cap, count, dump, status);
    return cudaGetLastError() == cudaSuccess ? DOG_OK : DOG_ERR_CUDA;
}

}  // namespace dogk
