// Device helpers shared by the detection kernels (sm_103a): the reflect
// boundary, pixel ingest and the DoG value, so that the fused kernel and the
// strip-edge resolve form every value with the same operations.
#pragma once

#include <cuda_runtime.h>

#include "dog.h"
#include "dog_internal.cuh"

namespace dogk {

// Half-sample-symmetric reflection of index i into [0, n): -1 -> 0,
// -k -> k-1, n+k -> n-1-k, folded with period 2n for any i.
__device__ __forceinline__ int refl(int i, int n) {
    if (i >= 0 && i < n) return i;
    int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m >= n ? p - 1 - m : m;
}

// v / d, correctly rounded, for integers |v| <= 4095 and 1 <= d <= 4095, from
// rd = RN(1/d): the product q = RN(v rd) and one FMA correction with the exact
// remainder v - q d (Markstein's final step, IBM J. Res. Dev. 34(1), 1990).
// Checked against the correctly rounded quotient for every such v >= 0 and d
// (the rounding is symmetric, so negative v follow); three instructions where
// the IEEE division routine takes many more.
__device__ __forceinline__ float div_small(float v, float d, float rd) {
    const float q = __fmul_rn(v, rd);
    const float rem = __fmaf_rn(-q, d, v);
    return __fmaf_rn(rem, rd, q);
}
constexpr float RCP_4095 = 1.0f / 4095.0f;   // RN(1/4095)

// Reciprocal of the stretch span hi - lo (0 when the limits are equal), once
// per tile or thread.
__device__ __forceinline__ float stretch_rcp(int lo, int hi) {
    return hi > lo ? __frcp_rn((float)(hi - lo)) : 0.0f;
}

// Contrast stretch of one count (Sec. 4 preprocessing): counts above 4095 act
// as 4095; (c - lo) / (hi - lo) correctly rounded (both operands are exact
// integers), clipped to [0, 1]; equal limits map to 0 at or below the limit
// and 1 above.  rcp = stretch_rcp(lo, hi).
__device__ __forceinline__ float stretch_px(unsigned v, int lo, int hi, float rcp) {
    const int c = min((int)v, STRETCH_BINS - 1);
    if (hi <= lo) return c > lo ? 1.0f : 0.0f;
    const float t = div_small((float)(c - lo), (float)(hi - lo), rcp);
    return fminf(fmaxf(t, 0.0f), 1.0f);
}

// Raw pixel load and its conversion to [0, 1] (uint16 counts: v / 4095
// correctly rounded, or the contrast stretch with limits lo, hi).
__device__ __forceinline__ unsigned load_raw(const void* img, int dtype, int pitch, int y, int x) {
    if (dtype != DOG_DTYPE_F32)
        return (unsigned)__ldg(reinterpret_cast<const unsigned short*>(img) + (size_t)y * pitch + x);
    return __float_as_uint(__ldg(reinterpret_cast<const float*>(img) + (size_t)y * pitch + x));
}
__device__ __forceinline__ float raw_to_px(unsigned v, int dtype, int lo, int hi, float rcp) {
    if (dtype == DOG_DTYPE_U16) return div_small((float)v, 4095.0f, RCP_4095);
    if (dtype == DTYPE_U16_STRETCH) return stretch_px(v, lo, hi, rcp);
    return __uint_as_float(v);
}

__device__ __forceinline__ float dog_value(float c, float a, float b) {
    return __fmul_rn(c, __fsub_rn(a, b));
}

}  // namespace dogk
