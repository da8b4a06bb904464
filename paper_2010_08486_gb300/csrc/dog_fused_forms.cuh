// Fused DoG detector kernel for sm_103a: the kernel forms, templated on the
// number of producer warps (dog_fused.cu and dog_fused_w8.cu instantiate them).
//
// Method (arXiv 2010.08486): scale space L_i = g(sigma_i) * I (Sec. 3), DoG
// D_i = c_i (L_i - L_{i+1}) (Eq. 2-3), voxels equal to their 3x3x3 maximum
// and above the threshold (Sec. 4, Sec. 4.1).
//
// Design.  A CTA owns a strip of TX = 32 output columns and walks down a
// band of rows in blocks of MB = 8 rows, so every input pixel of the strip
// is read once from global memory for all K scales and no vertical halo is
// recomputed.  Each producer warp owns a fixed set of levels, chosen on the
// host to balance taps (forms with 8 and with 12 producer warps; the host
// picks one per ladder).  For each block and owned level a warp
//   1. runs the horizontal pass of the next 8 input rows into the level's
//      circular shared-memory ring (which runs Tpad/8 blocks ahead),
//   2. runs the vertical pass over the ring into the block's L rows.
// Both passes are register-blocked 1-D correlations: 8 outputs per lane,
// taps in blocks of 8 against a two-window register file whose halves swap
// roles each block, so one short loop serves every radius and the whole
// kernel stays resident in the instruction cache.  Kernels are zero-padded to
// Tpad = 8 ceil((2r+1)/8) taps; taps are summed in ascending order with FMA
// from zero, so the padding never changes a value and the resolve kernel
// (dog_resolve.cu), which repeats the order on the real taps only, reproduces
// any response bit for bit.  Then all threads form D in place and test the
// previous block's rows against their 26 neighbours; survivors are compacted
// with one warp ballot and one atomic per warp.  Neighbours in the adjacent
// strip are not held here: in detection a candidate at a strip edge is
// queued and the resolve kernel recomputes the few responses it needs; the
// soft modes, which keep every local maximum (thousands at strip edges per
// frame), instead step 32-column strips by 30 so that lanes 0 and 31 are
// only neighbours and every voxel a strip owns has its whole neighbourhood.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "dog_internal.cuh"
#include "dog_device.cuh"

namespace dogk {

// ---------------------------------------------------------------------------
// 1-D passes.  out[k] = sum_{t=0}^{Tpad-1} wfull[t] * in[k+t], k = 0..7, in
// ascending t from 0.  A holds inputs [8j, 8j+8), B inputs [8j+8, 8j+16) of
// tap block j; the 64 products of the block are accumulated tap-major.
__device__ __forceinline__ void fma_block(float (&acc)[8], const float (&A)[8], const float (&B)[8],
                                          const float4 wa, const float4 wb) {
    const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = __fmaf_rn(w[u], (k + u < 8) ? A[k + u] : B[k + u - 8], acc[k]);
}

// The single last tap of a level whose 2r + 1 taps are one more than a
// multiple of 8 (the rest of its padded block is zeros): out[k] += w * Y[k],
// Y the window after the last full tap block.
__device__ __forceinline__ void tap1(float (&acc)[8], const float (&Y)[8], float w) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = __fmaf_rn(w, Y[k], acc[k]);
}

// Horizontal: inputs are consecutive floats of one shared-memory row.
// Output: 8 floats of one ring row, written as two float4 whose order is
// swapped on odd rows (bank swizzle; `odd` is the ring row's parity).
__device__ __forceinline__ void hpass(const float* __restrict__ src, float* __restrict__ dst, int odd,
                                      const float4* __restrict__ w4, int nb, bool tail) {
    float acc[8], A[8], B[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { acc[k] = 0.0f; A[k] = src[k]; }
    src += 8;
    for (;;) {
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = src[k];
        fma_block(acc, A, B, w4[0], w4[1]);
        if (--nb == 0) {
            if (tail) tap1(acc, B, w4[2].x);
            break;
        }
        src += 8;
        w4 += 2;
#pragma unroll
        for (int k = 0; k < 8; ++k) A[k] = src[k];
        fma_block(acc, B, A, w4[0], w4[1]);
        if (--nb == 0) {
            if (tail) tap1(acc, A, w4[2].x);
            break;
        }
        src += 8;
        w4 += 2;
    }
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4 lo = make_float4(acc[0], acc[1], acc[2], acc[3]);
    const float4 hi = make_float4(acc[4], acc[5], acc[6], acc[7]);
    d4[odd] = lo;
    d4[odd ^ 1] = hi;
}

// Vertical: inputs are rows of a circular ring of C rows (C a multiple of 8),
// read in blocks of 8 rows starting at ring row r0 (a multiple of 8); lane x
// holds column x, stored at x on even rows and x ^ 4 on odd rows.
__device__ __forceinline__ void vpass(const float* __restrict__ ring, int lane, int C, int r0,
                                      const float4* __restrict__ w4, int nb, bool tail, float (&acc)[8]) {
    const float* pe = ring + lane;
    const float* po = ring + (lane ^ 4);
    float A[8], B[8];
    int r = r0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k] = 0.0f;
        A[k] = ((k & 1) ? po : pe)[(r + k) * RING_STRIDE];
    }
    r += 8;
    if (r == C) r = 0;
    for (;;) {
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = ((k & 1) ? po : pe)[(r + k) * RING_STRIDE];
        fma_block(acc, A, B, w4[0], w4[1]);
        if (--nb == 0) {
            if (tail) tap1(acc, B, w4[2].x);
            break;
        }
        r += 8;
        if (r == C) r = 0;
        w4 += 2;
#pragma unroll
        for (int k = 0; k < 8; ++k) A[k] = ((k & 1) ? po : pe)[(r + k) * RING_STRIDE];
        fma_block(acc, B, A, w4[0], w4[1]);
        if (--nb == 0) {
            if (tail) tap1(acc, A, w4[2].x);
            break;
        }
        r += 8;
        if (r == C) r = 0;
        w4 += 2;
    }
}

// ---------------------------------------------------------------------------
struct TileCtx {
    const void* img;
    int dtype, H, W, pitch;
    int st_lo, st_hi;   // contrast-stretch limits (DTYPE_U16_STRETCH)
    float st_rcp;       // stretch_rcp(st_lo, st_hi)
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

// Named barriers (id 0 is __syncthreads).
//   FULL:  producers arrive once a block's L rows are written; consumers wait.
//   EMPTY: consumers arrive once a block's rows are no longer needed;
//          producers wait before overwriting them two blocks later.
//   PROD:  producers only, once per block (input-row visibility).
//   CONS:  consumers only, between forming D and testing.
// FULL and EMPTY alternate between two ids by block parity, so each id has at
// most one generation outstanding: a producer arrives at FULL(b+2) only after
// waiting EMPTY(b), which consumers signal after their wait on FULL(b), and
// consumers arrive at EMPTY(b+2) only after FULL(b+2), which producers signal
// after their wait on EMPTY(b).
enum { BAR_FULL = 1, BAR_EMPTY = 3, BAR_PROD = 5, BAR_CONS = 6 };

__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
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
    int rpos[MAX_LEVELS];     // ring row of each level's window start
    int tile;
    LevelInfo lv[MAX_LEVELS]; // per-level table (copied from the parameters once)
    int wn[NWARPS];           // levels owned by each producer warp
    unsigned char wl[NWARPS][MAX_LEVELS];
};

__device__ __forceinline__ int dslot(int k) { return k >= DSLOTS ? k - DSLOTS : k; }

// Producer warps: blur passes.  Block b's L rows go to DoG-buffer slots
// (8b + 2 + k) mod DSLOTS.
template <int NW>
__device__ __forceinline__ void produce(const FusedParams& p, float* sm, SmemSmall& ss, const TileCtx& tc, int emax,
                        int nblk) {
    constexpr int NTHREADS = (NW + NCONS) * 32, NPROD_T = NW * 32;
    const int tid = threadIdx.x;       // 0 .. NPROD_T-1
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int R = p.R;
    const int CIN = p.in_rows;        // input-buffer rows (a power of two)
    const int S = p.in_stride;
    const int ncols = TX + 2 * R;     // input columns per row (<= NPROD_T)
    const int yb0 = tc.y0 - 1;
    const int yorg = yb0 - MB * emax;   // input-ring slot origin
    float* in = sm + p.in_off;
    float* dbuf = sm + p.d_off;
    // producer warps 0 .. MB-1 each fetch one of the MB rows a block adds,
    // lane x columns x, x + 32, ... of the TX + 2R loaded ones
    static_assert(NW >= MB, "one prefetched row per producer warp");
    constexpr int NPF = (TX + 2 * DOG_MAX_RADIUS + 31) / 32;

    for (int b = -emax; b < nblk; ++b) {
        const int yb = yb0 + MB * b;
        // prefetch the 8 rows block b+1 adds (latency hidden behind the passes)
        unsigned pf[NPF];   // raw pixel bits; converted when stored, after the passes
        const int ynew = yorg + MB * (b + emax + 1) + p.dmax;
        const bool do_pf = b + 1 < nblk && warp < MB;
        const int yrow = refl(ynew + warp, tc.H);
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int cc = lane + 32 * k;
            pf[k] = (do_pf && cc < ncols) ? load_raw(tc.img, tc.dtype, tc.pitch, yrow, refl(tc.x0 - R + cc, tc.W)) : 0u;
        }
        // block b's L rows overwrite those of block b-2: wait for the consumers
        if (b >= 2) bar_sync(BAR_EMPTY + (b & 1), NTHREADS);

        const int nl = ss.wn[warp];
        const int s0 = b >= 0 ? (MB * b + 2) % DSLOTS : 0;   // DoG-buffer slot of row yb
        for (int li = 0; li < nl; ++li) {
            const int i = ss.wl[warp][li];
            const LevelInfo L = ss.lv[i];
            const int C = L.ring_rows;
            const int r0 = ss.rpos[i];     // 8b mod C; the chunk written now goes 8 rows before
            if (b + L.e >= 0) {
                float* ring = sm + L.ring_off;
                // 2r + 1 = 8 (nb - 1) + 1: nb - 1 full tap blocks and one last tap
                const bool tail = ((2 * L.r + 1) & 7) == 1;
                const int nb = (L.tpad >> 3) - (tail ? 1 : 0);
                {
                    const int rho = lane >> 2, g = lane & 3;
                    const int yy = yb + L.delta + rho;     // input row of this lane
                    const float* src = in + ((yy - yorg) & (CIN - 1)) * S + (R - L.r) + 8 * g;
                    const int wrow = (r0 >= MB ? r0 - MB : r0 + C - MB) + rho;
                    hpass(src, ring + wrow * RING_STRIDE + 8 * g, rho & 1,
                          reinterpret_cast<const float4*>(sm + p.w_off + L.hoff), nb, tail);
                }
                __syncwarp();
                if (b >= 0) {
                    float acc[8];
                    vpass(ring, lane, C, r0, reinterpret_cast<const float4*>(sm + p.w_off + L.woff), nb, tail, acc);
                    float* dcol = dbuf + i * DSLOTS * TX + lane;
#pragma unroll
                    for (int k = 0; k < 8; ++k) dcol[dslot(s0 + k) * TX] = acc[k];
                }
            }
            __syncwarp();
            if (lane == 0) ss.rpos[i] = (r0 + MB == C) ? 0 : r0 + MB;
        }
        // input rows of block b+1 (their slots are not read by block b)
        if (do_pf) {
            float* dst = in + ((ynew + warp - yorg) & (CIN - 1)) * S;
#pragma unroll
            for (int k = 0; k < NPF; ++k) {
                const int cc = lane + 32 * k;
                if (cc < ncols) dst[cc] = raw_to_px(pf[k], tc.dtype, tc.st_lo, tc.st_hi, tc.st_rcp);
            }
        }
        if (b >= 0) bar_arrive(BAR_FULL + (b & 1), NTHREADS);
        bar_sync(BAR_PROD, NPROD_T);
    }
}


// Consumer warps: the 3x3x3 test of rows yb-1 .. yb+6 (two rows per warp),
// with D_l = c_l (L_l - L_{l+1}) formed on the fly from the L rows the
// producers wrote (the DoG buffer is never rewritten).
//
// Plane loop of one test row y: returns the mask of planes l whose voxel
// (x, y, l) is a candidate: D_l(y, x) > thr and D_l(y, x) >= m_{l-1}, m_l,
// m_{l+1}, where m_j is the 3x3 maximum of plane j around (x, y) (-inf for
// planes outside the ladder).  Plane l - 1 is tested as soon as m_l exists,
// so only a window of three maxima is live.  The vertical maximum of
// c (L_l - L_{l+1}) over rows y-1 .. y+1 is formed as c max(L_l - L_{l+1}):
// c > 0 and rounding is monotonic, so both are the same number.  Lanes 0 and
// 31 receive their own value from the shuffles, which leaves their maximum
// unchanged: neighbours outside the strip are outside the frame (-inf) or
// settled by the resolve kernel.  EDGE: row y-1 or y+1 lies outside the
// frame, or the strip has columns past the frame's right edge (-inf there).
template <int PB, bool FULL, bool EDGE>
__device__ __forceinline__ unsigned test_planes(const float* colp, const float* cs, int P, int sm1, int sc, int sp1,
                                                bool ym_ok, bool yp_ok, bool col_ok, float thr) {
    const float NEG = -INFINITY;
    float m2 = NEG, m1 = NEG;   // 3x3 maxima of planes l-2, l-1
    float d1 = NEG;             // D_{l-1}(y, x)
    unsigned cmask = 0u;
    float Lu = colp[sm1 * TX], Lc = colp[sc * TX], Ld = colp[sp1 * TX];   // L_0 rows y-1, y, y+1
#pragma unroll
    for (int l = 0; l < PB; ++l) {
        const bool on = FULL || l < P;
        const float* pl = colp + (on ? l + 1 : P) * DSLOTS * TX;
        const float nu = pl[sm1 * TX], nc = pl[sc * TX], nd = pl[sp1 * TX];
        const float c = cs[l];
        const float eu = __fsub_rn(Lu, nu), ec = __fsub_rn(Lc, nc), en = __fsub_rn(Ld, nd);
        Lu = nu; Lc = nc; Ld = nd;
        const float d = __fmul_rn(c, ec);
        const float e = EDGE ? fmaxf(ec, fmaxf(ym_ok ? eu : NEG, yp_ok ? en : NEG)) : fmaxf(ec, fmaxf(eu, en));
        float m = __fmul_rn(c, e);
        m = (EDGE ? (on && col_ok) : on) ? m : NEG;
        const float ml = __shfl_up_sync(0xffffffffu, m, 1);
        const float mr = __shfl_down_sync(0xffffffffu, m, 1);
        const float m0 = fmaxf(m, fmaxf(ml, mr));
        if (l >= 1) {
            const bool cand = d1 >= fmaxf(m0, fmaxf(m2, m1)) && d1 > thr && (FULL || l - 1 < P);
            cmask |= cand ? (1u << (l - 1)) : 0u;
        }
        m2 = m1;
        m1 = m0;
        d1 = d;
    }
    const bool cand = d1 >= fmaxf(m2, m1) && d1 > thr && (FULL || PB - 1 < P);
    cmask |= cand ? (1u << (PB - 1)) : 0u;
    return cmask;
}

// Plane loop of two adjacent test rows ya, yb = ya + 1 at once: their
// 3x3 windows share rows ya and yb, so four L rows per plane serve both.  The
// same operations as test_planes, row by row, so the masks are identical.
// a_up / a_dn / b_up / b_dn: rows ya-1 / yb / ya / yb+1 lie inside the frame.
template <int PB, bool FULL, bool EDGE>
__device__ __forceinline__ void test_planes2(const float* colp, const float* cs, int P, int s0, int s1, int s2,
                                             int s3, bool a_up, bool a_dn, bool b_up, bool b_dn, bool col_ok,
                                             float thr, unsigned& cma, unsigned& cmb) {
    const float NEG = -INFINITY;
    float m2a = NEG, m1a = NEG, d1a = NEG, m2b = NEG, m1b = NEG, d1b = NEG;
    unsigned ca = 0u, cb = 0u;
    float L0 = colp[s0 * TX], L1 = colp[s1 * TX], L2 = colp[s2 * TX], L3 = colp[s3 * TX];
#pragma unroll
    for (int l = 0; l < PB; ++l) {
        const bool on = FULL || l < P;
        const float* pl = colp + (on ? l + 1 : P) * DSLOTS * TX;
        const float n0 = pl[s0 * TX], n1 = pl[s1 * TX], n2 = pl[s2 * TX], n3 = pl[s3 * TX];
        const float c = cs[l];
        const float e0 = __fsub_rn(L0, n0), e1 = __fsub_rn(L1, n1), e2 = __fsub_rn(L2, n2), e3 = __fsub_rn(L3, n3);
        L0 = n0; L1 = n1; L2 = n2; L3 = n3;
        const float da = __fmul_rn(c, e1), db = __fmul_rn(c, e2);
        const float mid = fmaxf(e1, e2);
        const float va = EDGE ? fmaxf(a_up ? e0 : NEG, a_dn ? mid : e1) : fmaxf(e0, mid);
        const float vb = EDGE ? fmaxf(b_up ? mid : e2, b_dn ? e3 : NEG) : fmaxf(mid, e3);
        const bool live = EDGE ? (on && col_ok) : on;
        const float ma = live ? __fmul_rn(c, va) : NEG;
        const float mb = live ? __fmul_rn(c, vb) : NEG;
        const float la = __shfl_up_sync(0xffffffffu, ma, 1), ra = __shfl_down_sync(0xffffffffu, ma, 1);
        const float lb = __shfl_up_sync(0xffffffffu, mb, 1), rb = __shfl_down_sync(0xffffffffu, mb, 1);
        const float m0a = fmaxf(ma, fmaxf(la, ra)), m0b = fmaxf(mb, fmaxf(lb, rb));
        if (l >= 1) {
            const bool okl = FULL || l - 1 < P;
            ca |= (d1a >= fmaxf(m0a, fmaxf(m2a, m1a)) && d1a > thr && okl) ? (1u << (l - 1)) : 0u;
            cb |= (d1b >= fmaxf(m0b, fmaxf(m2b, m1b)) && d1b > thr && okl) ? (1u << (l - 1)) : 0u;
        }
        m2a = m1a; m1a = m0a; d1a = da;
        m2b = m1b; m1b = m0b; d1b = db;
    }
    const bool okl = FULL || PB - 1 < P;
    ca |= (d1a >= fmaxf(m2a, m1a) && d1a > thr && okl) ? (1u << (PB - 1)) : 0u;
    cb |= (d1b >= fmaxf(m2b, m1b) && d1b > thr && okl) ? (1u << (PB - 1)) : 0u;
    cma = ca;
    cmb = cb;
}

// D_l(y, x) of the test row (slot sc), recomputed for a candidate with the
// operations of the plane loop.
__device__ __forceinline__ float d_at(const float* colp, const float* cs, int l, int sc) {
    return dog_value(cs[l], colp[l * DSLOTS * TX + sc * TX], colp[(l + 1) * DSLOTS * TX + sc * TX]);
}

// Per test row y and plane l: D at rows y-1, y, y+1 (three loads of L_{l+1},
// the L_l rows carried from plane l-1), its vertical maximum, then the
// horizontal maximum through two warp shuffles -> m_l; a voxel is a
// candidate iff D_l(y, x) >= max(m_{l-1}, m_l, m_{l+1}) (it equals its 3x3x3
// maximum).  Neighbours outside the frame count as -inf; those in the
// adjacent strip are left to the resolve kernel (the candidate is queued),
// unless the strips overlap (soft modes).
// The plane loop is unrolled over PB >= P planes without branches (planes
// l >= P read plane P and are masked to -inf), keeping m and D in registers;
// candidates are collected in a per-lane bit mask and compacted afterwards
// (they are rare).
template <int NW, bool BATCHED, int PB, bool FULL>
__device__ __forceinline__ void consume(const FusedParams& p, float* sm, SmemSmall& ss, const TileCtx& tc, int nblk) {
    constexpr int NTHREADS = (NW + NCONS) * 32;
    const int cw = (threadIdx.x >> 5) - NW;   // 0 .. NCONS-1
    const int lane = threadIdx.x & 31;
    const int P = p.P;
    const int yb0 = tc.y0 - 1;
    const float* dbuf = sm + p.d_off;
    const int mode = p.mode;
    const bool soft = (mode == MODE_SOFT || mode == MODE_BWD);
    const float thr = soft ? -INFINITY : p.thr;   // D > thr is not applied to soft maxima
    const int x = lane;
    const int gx = tc.x0 + x;
    const bool col_ok = gx >= 0 && gx < tc.W;   // a real column (neighbours of owned voxels)
    // voxels this lane settles: with overlapping strips lanes 0 and TX-1 are
    // only neighbours (the adjacent strips own those columns); otherwise a
    // strip-edge voxel whose neighbours lie in the adjacent strip is queued
    const bool overlap = !BATCHED && p.overlap;   // (single-frame launches only)
    const bool own = col_ok && (!overlap || (x >= 1 && x <= TX - 2));
    const bool edge_x = !overlap && ((x == 0 && tc.x0 > 0) || (x == TX - 1 && gx + 1 < tc.W));
    const float* colp = dbuf + x;

    for (int b = 0; b < nblk; ++b) {
        const int yb = yb0 + MB * b;
        bar_sync(BAR_FULL + (b & 1), NTHREADS);
        // two rows per consumer warp: both masks from one plane loop
        unsigned cm2a = 0u, cm2b = 0u;
        if (MB / NCONS == 2 && mode != MODE_DUMP) {
            const int wa = cw * 2;
            const int ya = yb - 1 + wa;
            const int s0 = (MB * b + wa) % DSLOTS, s1 = (MB * b + wa + 1) % DSLOTS;
            const int s2 = (MB * b + wa + 2) % DSLOTS, s3 = (MB * b + wa + 3) % DSLOTS;
            const bool a_up = ya - 1 >= 0, a_dn = ya + 1 < tc.H, b_up = ya >= 0, b_dn = ya + 2 < tc.H;
            if (a_up && b_dn && tc.x0 >= 0 && tc.x0 + TX <= tc.W)
                test_planes2<PB, FULL, false>(colp, ss.c, P, s0, s1, s2, s3, a_up, a_dn, b_up, b_dn, col_ok, thr,
                                              cm2a, cm2b);
            else
                test_planes2<PB, FULL, true>(colp, ss.c, P, s0, s1, s2, s3, a_up, a_dn, b_up, b_dn, col_ok, thr,
                                             cm2a, cm2b);
        }
#pragma unroll 1
        for (int q = 0; q < MB / NCONS; ++q) {
            const int w = cw * (MB / NCONS) + q;
            const int y = yb - 1 + w;
            const bool row_ok = (y >= tc.y0 && y < tc.y1);
            const int sc = (MB * b + w + 1) % DSLOTS;    // slot of row y
            const int sm1 = (MB * b + w) % DSLOTS;       // row y-1
            const int sp1 = (MB * b + w + 2) % DSLOTS;   // row y+1
            const bool ym_ok = y - 1 >= 0, yp_ok = y + 1 < tc.H;
            if (mode == MODE_DUMP) {
                if (row_ok && own) {
                    for (int l = 0; l < P; ++l) {
                        const float* pl = colp + l * DSLOTS * TX;
                        p.dump[((size_t)l * tc.H + y) * tc.W + gx] =
                            dog_value(ss.c[l], pl[sc * TX], pl[DSLOTS * TX + sc * TX]);
                    }
                }
                continue;
            }
            unsigned cmask;
            if (MB / NCONS == 2)
                cmask = q == 0 ? cm2a : cm2b;
            else if (ym_ok && yp_ok && tc.x0 + TX <= tc.W)
                cmask = test_planes<PB, FULL, false>(colp, ss.c, P, sm1, sc, sp1, ym_ok, yp_ok, col_ok, thr);
            else
                cmask = test_planes<PB, FULL, true>(colp, ss.c, P, sm1, sc, sp1, ym_ok, yp_ok, col_ok, thr);
            if (!(row_ok && own)) cmask = 0u;
            const unsigned dmask = edge_x ? 0u : cmask;   // settled here
            const unsigned pmask = edge_x ? cmask : 0u;   // queued for the resolve kernel
            // ---- queued strip-edge candidates (lanes 0 and 31 only)
            if (__any_sync(0xffffffffu, pmask != 0u)) {
                unsigned rest = pmask;
                while (rest) {
                    const int l = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const int idx = atomicAdd(p.pend_count, 1);
                    if (idx < p.pend_cap) {
                        Pending e;
                        e.frame = tc.frame; e.x = gx; e.y = y; e.level = l; e.response = d_at(colp, ss.c, l, sc);
                        p.pend[idx] = e;
                    } else {
                        atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                    }
                }
            }
            if (mode == MODE_CANDIDATES) {
                // one warp-wide slot reservation for all the row's candidates
                const int nmine = __popc(dmask);
                int incl = nmine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                if (total) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(tc.count, total);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    int idx = base + incl - nmine;
                    unsigned rest = dmask;
                    while (rest) {
                        const int l = __ffs(rest) - 1;
                        rest &= rest - 1;
                        if (idx < p.cap) {
                            dog_blob bl;
                            bl.x = gx; bl.y = y; bl.level = l; bl.sigma = ss.sig[l]; bl.response = d_at(colp, ss.c, l, sc);
                            tc.blobs[idx] = bl;
                        } else {
                            atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                        }
                        ++idx;
                    }
                }
            } else if (mode == MODE_SOFT) {
                // optional record of the maxima for the backward: each lane
                // with maxima reserves its slots (about one lane per warp row)
                int idx = 0;
                if (p.rec != nullptr && dmask != 0u) idx = atomicAdd(p.rec_count, __popc(dmask));
                unsigned rest = dmask;
                while (rest) {
                    const int l = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const float e = __fsub_rn(colp[l * DSLOTS * TX + sc * TX], colp[(l + 1) * DSLOTS * TX + sc * TX]);
                    const float d = __fmul_rn(ss.c[l], e);   // = d_at(colp, ss.c, l, sc)
                    const float s = 1.0f / (1.0f + __expf(-(d - p.thr) * p.inv_T));
                    atomicAdd(&ss.soft[ss.kb[l][0]], s * ss.kw[l][0]);
                    atomicAdd(&ss.soft[ss.kb[l][1]], s * ss.kw[l][1]);
                    if (p.rec != nullptr) {
                        if (idx < p.rec_cap) {
                            const float q = s * (1.0f - s) * p.inv_T;
                            dog_soft_max m;
                            m.x = gx; m.y = y; m.level = l; m.q = q; m.qe = q * e; m.s = s;
                            p.rec[idx] = m;
                        } else {
                            atomicCAS(p.status, 0, (int)DOG_ERR_CAPACITY);
                        }
                        ++idx;
                    }
                }
            } else {
                // backward prologue: dense dloss/dL rows A_l = c_l G_l - c_{l-1} G_{l-1}
                float Gprev = 0.0f;
#pragma unroll
                for (int l = 0; l < PB; ++l) {
                    if (l < P) {
                        float G = 0.0f;
                        if (dmask & (1u << l)) {
                            const float d = d_at(colp, ss.c, l, sc);
                            const float s = 1.0f / (1.0f + __expf(-(d - p.thr) * p.inv_T));
                            G = ss.gk[l] * s * (1.0f - s) * p.inv_T;
                            atomicAdd(&ss.dc[l], G * d / ss.c[l]);
                            atomicAdd(&ss.dt[l], s * ss.gdk[l]);
                        }
                        if (row_ok && own) {
                            p.A[((size_t)l * tc.H + y) * tc.W + gx] = ss.c[l] * G - (l > 0 ? ss.c[l - 1] * Gprev : 0.0f);
                            if (l == P - 1) p.A[((size_t)(l + 1) * tc.H + y) * tc.W + gx] = -ss.c[l] * G;
                        }
                        Gprev = G;
                    }
                }
            }
        }
        // rows yb-2 .. yb+5 are free for block b+2 (arrivals match the producers' waits)
        if (b + 2 < nblk) bar_arrive(BAR_EMPTY + (b & 1), NTHREADS);
    }
}

template <int NW, bool BATCHED, int PB, bool FULL>
__device__ __forceinline__ void process_tile(const FusedParams& p, float* sm, SmemSmall& ss, const TileCtx& tc) {
    constexpr int NTHREADS = (NW + NCONS) * 32, NPROD_T = NW * 32;
    const int tid = threadIdx.x;
    const int yb0 = tc.y0 - 1;
    const int nblk = (tc.y1 - tc.y0 + 2 + MB - 1) / MB;
    int emax = 0;
    for (int i = 0; i < p.K; ++i) emax = max(emax, ss.lv[i].e);
    const int yorg = yb0 - MB * emax;
    const int R = p.R;
    const int ncols = TX + 2 * R;
    // initial input rows (those read at block -emax), spread over all threads;
    // each thread issues its loads before converting and storing any
    float* in = sm + p.in_off;
    {
        const int y0 = yorg + p.dmin;
        const int total = (p.dmax + MB - p.dmin) * ncols;
        for (int i0 = 0; i0 < total; i0 += 8 * NTHREADS) {
            unsigned v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NTHREADS + tid;
                v[u] = 0u;
                if (i < total) {
                    const int rr = i / ncols, cc = i - rr * ncols;
                    v[u] = load_raw(tc.img, tc.dtype, tc.pitch, refl(y0 + rr, tc.H), refl(tc.x0 - R + cc, tc.W));
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NTHREADS + tid;
                if (i < total) {
                    const int rr = i / ncols, cc = i - rr * ncols;
                    in[((y0 + rr - yorg) & (p.in_rows - 1)) * p.in_stride + cc] =
                        raw_to_px(v[u], tc.dtype, tc.st_lo, tc.st_hi, tc.st_rcp);
                }
            }
        }
    }
    for (int i = tid; i < p.K; i += NTHREADS) {
        const int C = ss.lv[i].ring_rows;
        ss.rpos[i] = ((-MB * emax) % C + C) % C;
    }
    __syncthreads();
    if (tid < NPROD_T) produce<NW>(p, sm, ss, tc, emax, nblk);
    else consume<NW, BATCHED, PB, FULL>(p, sm, ss, tc, nblk);
    __syncthreads();
}

template <int NW, bool BATCHED, int PB, bool FULL>
__global__ void __launch_bounds__((NW + NCONS) * 32, 1) dog_fused_kernel(const __grid_constant__ FusedParams p) {
    constexpr int NTHREADS = (NW + NCONS) * 32;
    extern __shared__ float4 dyn4[];
    float* sm = reinterpret_cast<float*>(dyn4);
    __shared__ SmemSmall ss;
    const int tid = threadIdx.x;
    // zero the dynamic shared memory once: zero-weight padding taps may read
    // input-row columns past the loaded ones, and those must be finite
    for (int q = tid; q < p.smem_bytes / 16; q += NTHREADS) dyn4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int q = tid; q < p.w_total; q += NTHREADS) sm[p.w_off + q] = p.w[q];
    for (int q = tid; q < MAX_LEVELS; q += NTHREADS) ss.c[q] = q < p.P ? p.c[q] : 0.0f;
    for (int q = tid; q < p.K; q += NTHREADS) ss.lv[q] = p.lv[q];
    for (int q = tid; q < NWARPS * MAX_LEVELS; q += NTHREADS) ss.wl[q / MAX_LEVELS][q % MAX_LEVELS] =
        p.warp_lev[q / MAX_LEVELS][q % MAX_LEVELS];
    for (int q = tid; q < NWARPS; q += NTHREADS) ss.wn[q] = p.warp_nlev[q];
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
        tc.st_lo = tc.dtype == DTYPE_U16_STRETCH ? p.lohi[0] : 0;
        tc.st_hi = tc.dtype == DTYPE_U16_STRETCH ? p.lohi[1] : 0;
        tc.st_rcp = stretch_rcp(tc.st_lo, tc.st_hi);
        const int strip = blockIdx.x % p.n_strips;
        const int band = blockIdx.x / p.n_strips;
        tc.x0 = p.overlap ? strip * (TX - 2) - 1 : strip * TX;
        tc.y0 = band * p.band;
        tc.y1 = min(p.H, tc.y0 + p.band);
        tc.blobs = p.blobs;
        tc.count = p.count;
        process_tile<NW, BATCHED, PB, FULL>(p, sm, ss, tc);
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
            tc.st_lo = tc.dtype == DTYPE_U16_STRETCH ? p.lohi[2 * lo] : 0;
            tc.st_hi = tc.dtype == DTYPE_U16_STRETCH ? p.lohi[2 * lo + 1] : 0;
            tc.st_rcp = stretch_rcp(tc.st_lo, tc.st_hi);
            tc.x0 = (local % f.n_strips) * TX;
            const int band = local / f.n_strips;
            const int bh = f.band;
            tc.y0 = band * bh;
            tc.y1 = min(f.h, tc.y0 + bh);
            tc.blobs = p.blobs + f.blob_off;
            tc.count = p.count + lo;
            process_tile<NW, BATCHED, PB, FULL>(p, sm, ss, tc);
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

// The dynamic shared-memory limit is raised once per device and kernel form
// (not on every launch, so launches can be captured into CUDA graphs); atomic
// because handles on other host threads launch the same forms.
static std::atomic<int> g_smem_limit[64][16];

template <int NW, bool BATCHED, int PB, bool FULL>
static cudaError_t launch_form(const FusedParams& p, int grid, cudaStream_t s, std::atomic<int>* lim) {
    if (lim->load(std::memory_order_acquire) < p.smem_bytes) {
        cudaError_t e = cudaFuncSetAttribute(dog_fused_kernel<NW, BATCHED, PB, FULL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
        if (e != cudaSuccess) return e;
        int cur = lim->load(std::memory_order_relaxed);
        while (cur < p.smem_bytes && !lim->compare_exchange_weak(cur, p.smem_bytes)) {
        }
    }
    dog_fused_kernel<NW, BATCHED, PB, FULL><<<grid, (NW + NCONS) * 32, p.smem_bytes, s>>>(p);
    return cudaGetLastError();
}

template <int NW, bool BATCHED, int PB>
static cudaError_t launch_bucket(const FusedParams& p, int grid, cudaStream_t s, std::atomic<int>* lim) {
    return p.P == PB ? launch_form<NW, BATCHED, PB, true>(p, grid, s, lim + 1)
                     : launch_form<NW, BATCHED, PB, false>(p, grid, s, lim);
}

// Plane-count buckets of the consumer's unrolled test: the smallest of 8, 16,
// 24 and MAX_LEVELS - 1 that holds P; a ladder that fills its bucket exactly
// runs a form without the masks of planes past the ladder.
template <int NW, bool BATCHED>
static cudaError_t launch_planes(const FusedParams& p, int grid, cudaStream_t s, std::atomic<int>* lim) {
    if (p.P <= 8) return launch_bucket<NW, BATCHED, 8>(p, grid, s, lim + 0);
    if (p.P <= 16) return launch_bucket<NW, BATCHED, 16>(p, grid, s, lim + 2);
    if (p.P <= 24) return launch_bucket<NW, BATCHED, 24>(p, grid, s, lim + 4);
    return launch_bucket<NW, BATCHED, MAX_LEVELS - 1>(p, grid, s, lim + 6);
}

// All forms of one producer-warp count (each translation unit instantiates one).
template <int NW>
static cudaError_t launch_fused_form(const FusedParams& p, int grid, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::atomic<int>* lim = g_smem_limit[dev & 63];
    return p.frames != nullptr ? launch_planes<NW, true>(p, grid, s, lim + 8)
                               : launch_planes<NW, false>(p, grid, s, lim);
}

}  // namespace dogk
