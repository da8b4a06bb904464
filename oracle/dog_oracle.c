/*
 * FP64 CPU oracle for Difference-of-Gaussians blob detection
 * (arXiv 2010.08486, "Towards Online Steering of Flame Spray Pyrolysis
 * Nanoparticle Synthesis", Sec. 3 and Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the detector computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the product path
 * never calls it, and it shares no code, header or table with the CUDA path.
 *
 * Every floating-point step is IEEE double.  Loops follow the definitions
 * literally; OpenMP only splits independent output elements across threads,
 * so results do not depend on the thread count.
 *
 * Readings of points the paper leaves open (each one is listed with its
 * justification in the design notes of the repository):
 *   - sigma ladder: geometric sigma_i = min * ratio^i, or Eq. 1 literally;
 *   - sign: D_i = c_i (L_i - L_{i+1}) so that bright blobs respond positively
 *     (Sec. 3 states the dark/bright convention; the threshold test of
 *     Sec. 4.1 keeps D > 0.1);
 *   - c_i = sigma_i / (sigma_{i+1} - sigma_i) ("DERIV", the finite-difference
 *     form of the heat-equation identity in Sec. 3) or c_i = sigma_i (Eq. 3
 *     literally, "PAPER");
 *   - radius_i = floor(truncate * sigma_i + 0.5) (Sec. 4.1 gives
 *     radius = truncate * sigma), point-sampled kernel normalised to sum 1;
 *   - boundary: half-sample symmetric reflection, folded repeatedly;
 *   - local maximum: D equals the 3x3x3 maximum filter, out-of-range
 *     neighbours ignored, strict threshold D > thr (Sec. 4, Sec. 4.1);
 *   - pruning: greedy coalescing in response order with the normalised
 *     lens overlap of the two circles r = sqrt(2) sigma (Sec. 4.1);
 *   - histogram: 32 bins on log volume between the first and last DoG plane.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_LADDER_GEOM 0
#define ORA_LADDER_ARITH 1
#define ORA_NORM_DERIV 0
#define ORA_NORM_PAPER 1
#define ORA_PRUNE_COALESCE 0
#define ORA_PRUNE_SUPPRESS 1
#define ORA_PRUNE_OFF 2
#define ORA_HIST_LOGV 0
#define ORA_HIST_LADDER 1

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Half-sample symmetric reflection of index i into [0, n): ... 2 1 0 | 0 1 2 ...
 * n-1 | n-1 n-2 ..., folded with period 2n so any offset maps in range. */
long ora_reflect(long i, long n) {
    long p = 2 * n;
    long m = i % p;
    if (m < 0) m += p;
    if (m >= n) m = p - 1 - m;
    return m;
}

/* Number of Gaussian levels of a geometric ladder that starts at min_sigma and
 * whose DoG planes reach max_sigma: k = floor(ln(max/min)/ln(ratio)) + 1 extra
 * steps, i.e. k + 1 levels (Sec. 4, n_bin + 1 kernels). */
int ora_ladder_geom_count(double min_sigma, double max_sigma, double ratio) {
    double steps = floor(log(max_sigma / min_sigma) / log(ratio) + 1e-9);
    return (int)steps + 2;
}

/* Geometric ladder sigma_i = min_sigma * ratio^i, i = 0..K-1. */
void ora_ladder_geom(double min_sigma, double ratio, int K, double* out) {
    for (int i = 0; i < K; ++i) out[i] = min_sigma * pow(ratio, (double)i);
}

/* Eq. 1: delta = (max - min) / n_bin, sigma_i = min + (i-1) delta for
 * i = 1..n_bin+1 (0-based here: sigma_i = min + i delta, K = n_bin + 1). */
void ora_ladder_arith(double min_sigma, double max_sigma, int K, double* out) {
    int n_bin = K - 1;
    double delta = (max_sigma - min_sigma) / (double)n_bin;
    for (int i = 0; i < K; ++i) out[i] = min_sigma + (double)i * delta;
}

/* Sec. 4.1: radius = truncate * sigma, rounded half up to an integer. */
int ora_radius(double sigma, double truncate) {
    return (int)floor(truncate * sigma + 0.5);
}

/* Sampled mean-zero Gaussian g(j, sigma) on j = -r..r, normalised to sum 1
 * (Sec. 3: L = g * I with g the Gaussian of standard deviation sigma). */
void ora_gauss_kernel(double sigma, int r, double* w) {
    double z = 0.0;
    for (int j = -r; j <= r; ++j) {
        double e = exp(-((double)j * (double)j) / (2.0 * sigma * sigma));
        w[j + r] = e;
        z += e;
    }
    for (int j = -r; j <= r; ++j) w[j + r] /= z;
}

/* d w_j / d sigma of the normalised kernel above with r held fixed:
 * w_j = e_j / Z, d e_j / d sigma = e_j j^2 / sigma^3, so
 * dw_j = w_j (j^2 - sum_k w_k k^2) / sigma^3. */
void ora_gauss_kernel_dsigma(double sigma, int r, double* dw) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(2 * r + 1));
    ora_gauss_kernel(sigma, r, w);
    double m2 = 0.0;
    for (int j = -r; j <= r; ++j) m2 += w[j + r] * (double)j * (double)j;
    double s3 = sigma * sigma * sigma;
    for (int j = -r; j <= r; ++j) dw[j + r] = w[j + r] * ((double)j * (double)j - m2) / s3;
    free(w);
}

/* Separable 2-D correlation with kernel kx along x (rows) then ky along y
 * (columns), both of radius r, under the reflect boundary:
 * out[y][x] = sum_a ky[a] sum_b kx[b] img[refl(y+a)][refl(x+b)]. */
void ora_blur2(const double* img, int h, int w, const double* kx, const double* ky, int r,
               double* out) {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)h * (size_t)w);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double s = 0.0;
            for (int b = -r; b <= r; ++b) s += kx[b + r] * img[(size_t)y * w + ora_reflect(x + b, w)];
            tmp[(size_t)y * w + x] = s;
        }
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double s = 0.0;
            for (int a = -r; a <= r; ++a) s += ky[a + r] * tmp[(size_t)ora_reflect(y + a, h) * w + x];
            out[(size_t)y * w + x] = s;
        }
    }
    free(tmp);
}

/* Scale-space level L(x, y, sigma) = g(sigma) * I (Sec. 3). */
void ora_blur(const double* img, int h, int w, double sigma, int r, double* out) {
    double* k = (double*)malloc(sizeof(double) * (size_t)(2 * r + 1));
    ora_gauss_kernel(sigma, r, k);
    ora_blur2(img, h, w, k, k, r, out);
    free(k);
}

/* Exact transpose of ora_blur2: every product that the forward gathers into
 * out[y][x] is scattered back onto the input pixel it read. */
void ora_blur2_adjoint(const double* a, int h, int w, const double* kx, const double* ky, int r,
                       double* grad) {
    double* tmp = (double*)calloc((size_t)h * (size_t)w, sizeof(double));
    /* transpose of the column pass: tmp[refl(y+a)][x] += ky[a] * a[y][x] */
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int q = -r; q <= r; ++q)
                tmp[(size_t)ora_reflect(y + q, h) * w + x] += ky[q + r] * a[(size_t)y * w + x];
    /* transpose of the row pass: grad[y][refl(x+b)] += kx[b] * tmp[y][x] */
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int b = -r; b <= r; ++b)
                grad[(size_t)y * w + ora_reflect(x + b, w)] += kx[b + r] * tmp[(size_t)y * w + x];
    free(tmp);
}

/* Scale normalisation c_i of plane i (Eq. 3 and the heat-equation argument of
 * Sec. 3): DERIV c_i = sigma_i / (sigma_{i+1} - sigma_i); PAPER c_i = sigma_i. */
void ora_norm_coeffs(const double* sig, int K, int norm, double* c) {
    for (int i = 0; i + 1 < K; ++i)
        c[i] = (norm == ORA_NORM_PAPER) ? sig[i] : sig[i] / (sig[i + 1] - sig[i]);
}

/* Eq. 2 and Eq. 3 with the sign read so that bright blobs are positive:
 * D_i = c_i (L_i - L_{i+1}), i = 0..K-2; D is (K-1) x h x w. */
void ora_dog(const double* img, int h, int w, const double* sig, const int* radii, int K,
             int norm, double* D) {
    size_t plane = (size_t)h * (size_t)w;
    double* L = (double*)malloc(sizeof(double) * plane * (size_t)K);
    double* c = (double*)malloc(sizeof(double) * (size_t)K);
    for (int i = 0; i < K; ++i) ora_blur(img, h, w, sig[i], radii[i], L + plane * (size_t)i);
    ora_norm_coeffs(sig, K, norm, c);
    for (int i = 0; i + 1 < K; ++i)
        for (size_t p = 0; p < plane; ++p)
            D[plane * (size_t)i + p] = c[i] * (L[plane * (size_t)i + p] - L[plane * (size_t)(i + 1) + p]);
    free(c);
    free(L);
}

/* Sec. 4 / Sec. 4.1: voxel v = (l, y, x) is a local maximum when it equals the
 * 3x3x3 maximum filter, i.e. no in-range neighbour is larger.  With use_thr it
 * must also exceed thr strictly.  Writes (l, y, x) triples and the response,
 * in ascending (l, y, x) order; returns the total count (may exceed cap). */
int ora_local_max(const double* D, int P, int h, int w, double thr, int use_thr,
                  int32_t* out_lyx, double* out_resp, int cap) {
    size_t plane = (size_t)h * (size_t)w;
    int n = 0;
    for (int l = 0; l < P; ++l)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double d = D[plane * (size_t)l + (size_t)y * w + x];
                if (use_thr && !(d > thr)) continue;
                int is_max = 1;
                for (int dl = -1; dl <= 1 && is_max; ++dl)
                    for (int dy = -1; dy <= 1 && is_max; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int ll = l + dl, yy = y + dy, xx = x + dx;
                            if (ll < 0 || ll >= P || yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                            if (D[plane * (size_t)ll + (size_t)yy * w + xx] > d) { is_max = 0; break; }
                        }
                if (!is_max) continue;
                if (n < cap) {
                    out_lyx[3 * n + 0] = l;
                    out_lyx[3 * n + 1] = y;
                    out_lyx[3 * n + 2] = x;
                    out_resp[n] = d;
                }
                ++n;
            }
    return n;
}

/* Normalised overlap of two discs: area of their intersection divided by the
 * area of the smaller disc.  1 when one contains the other, 0 when they are
 * disjoint; otherwise the two circular-segment areas of the lens. */
double ora_overlap(double x1, double y1, double r1, double x2, double y2, double r2) {
    double dx = x1 - x2, dy = y1 - y2;
    double d = sqrt(dx * dx + dy * dy);
    double rmin = r1 < r2 ? r1 : r2;
    if (d >= r1 + r2) return 0.0;
    if (d <= fabs(r1 - r2)) return 1.0;
    double c1 = (d * d + r1 * r1 - r2 * r2) / (2.0 * d * r1);
    double c2 = (d * d + r2 * r2 - r1 * r1) / (2.0 * d * r2);
    if (c1 > 1.0) c1 = 1.0;
    if (c1 < -1.0) c1 = -1.0;
    if (c2 > 1.0) c2 = 1.0;
    if (c2 < -1.0) c2 = -1.0;
    double k = (-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2);
    if (k < 0.0) k = 0.0;
    double area = r1 * r1 * acos(c1) + r2 * r2 * acos(c2) - 0.5 * sqrt(k);
    return area / (M_PI * rmin * rmin);
}

typedef struct { int32_t x, y, level; double resp; int idx; } ora_cand;

/* Priority: larger response first; equal responses by (level, y, x). */
static int ora_cand_cmp(const void* pa, const void* pb) {
    const ora_cand* a = (const ora_cand*)pa;
    const ora_cand* b = (const ora_cand*)pb;
    if (a->resp > b->resp) return -1;
    if (a->resp < b->resp) return 1;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

/* Sec. 4.1 pruning: blobs whose normalised overlap exceeds overlap_thr are
 * coalesced by averaging the radius.  Candidates are visited in priority
 * order; each joins the first blob accepted so far (in acceptance order) that
 * it overlaps, judged with both blobs' own ladder sigma, or is accepted.
 * COALESCE: an accepted blob reports the mean sigma of its group, summed in
 * visiting order (its own level's sigma exactly when every member shares that
 * level).  SUPPRESS: joiners are dropped.  OFF: every candidate passes.
 * r = sqrt(2) sigma (Sec. 4).  Output in acceptance order; returns count. */
int ora_prune(int n, const int32_t* x, const int32_t* y, const int32_t* level,
              const double* resp, const double* sig_ladder, double overlap_thr, int mode,
              int32_t* ox, int32_t* oy, int32_t* olevel, double* osigma, double* oresp) {
    ora_cand* c = (ora_cand*)malloc(sizeof(ora_cand) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        c[i].x = x[i]; c[i].y = y[i]; c[i].level = level[i]; c[i].resp = resp[i]; c[i].idx = i;
    }
    qsort(c, (size_t)n, sizeof(ora_cand), ora_cand_cmp);
    int* acc = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));     /* accepted -> c index */
    double* gsum = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int* gcnt = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* gmixed = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int na = 0;
    for (int i = 0; i < n; ++i) {
        int joined = -1;
        if (mode != ORA_PRUNE_OFF) {
            double si = sig_ladder[c[i].level];
            for (int a = 0; a < na; ++a) {
                const ora_cand* ca = &c[acc[a]];
                double sa = sig_ladder[ca->level];
                double ov = ora_overlap((double)c[i].x, (double)c[i].y, sqrt(2.0) * si,
                                        (double)ca->x, (double)ca->y, sqrt(2.0) * sa);
                if (ov > overlap_thr) { joined = a; break; }
            }
        }
        if (joined < 0) {
            acc[na] = i;
            gsum[na] = sig_ladder[c[i].level];
            gcnt[na] = 1;
            gmixed[na] = 0;
            ++na;
        } else if (mode == ORA_PRUNE_COALESCE) {
            gsum[joined] += sig_ladder[c[i].level];
            gcnt[joined] += 1;
            if (c[i].level != c[acc[joined]].level) gmixed[joined] = 1;
        }
    }
    for (int a = 0; a < na; ++a) {
        const ora_cand* ca = &c[acc[a]];
        ox[a] = ca->x;
        oy[a] = ca->y;
        olevel[a] = ca->level;
        osigma[a] = gmixed[a] ? gsum[a] / (double)gcnt[a] : sig_ladder[ca->level];
        oresp[a] = ca->resp;
    }
    free(gmixed);
    free(gcnt);
    free(gsum);
    free(acc);
    free(c);
    return na;
}

/* Blob volume from Sec. 4: r = sqrt(2) sigma, V = 4/3 pi r^3. */
double ora_volume(double sigma) {
    double r = sqrt(2.0) * sigma;
    return 4.0 / 3.0 * M_PI * r * r * r;
}

/* Histogram bin of one blob.  The blob's sigma is the value stored in the
 * blob record (single precision).  A blob whose stored sigma equals its
 * level's ladder sigma (rounded to single) is on the ladder: its bin comes
 * from its level alone, exactly: LOGV on a geometric ladder gives
 * floor(nbins * l / (K-2)) by integer arithmetic because ln V is affine in
 * the level; other ladders use the double formula on the ladder sigma.  Any
 * other sigma uses bin = floor(nbins (ln V - lo) / (hi - lo)) with lo, hi the
 * log volumes of the first and last DoG plane (LOGV), or the nearest ladder
 * plane in log sigma (LADDER, nbins = K-1).  Clamped to [0, nbins-1]. */
int ora_bin(float sigma_f32, int level, const double* sig_ladder, int K, int geom, int nbins,
            int mode) {
    int P = K - 1;
    int on_ladder = (sigma_f32 == (float)sig_ladder[level]);
    int b;
    if (mode == ORA_HIST_LADDER) {
        if (on_ladder) {
            b = level;
        } else {
            double ls = log((double)sigma_f32);
            int best = 0;
            double bd = fabs(ls - log(sig_ladder[0]));
            for (int l = 1; l < P; ++l) {
                double d = fabs(ls - log(sig_ladder[l]));
                if (d < bd) { bd = d; best = l; }
            }
            b = best;
        }
        nbins = P;
    } else {
        if (on_ladder && geom && P >= 2) {
            b = (int)(((long)nbins * (long)level) / (long)(P - 1));
        } else {
            double s = on_ladder ? sig_ladder[level] : (double)sigma_f32;
            double lo = log(ora_volume(sig_ladder[0]));
            double hi = log(ora_volume(sig_ladder[P - 1]));
            double t = (P >= 2 && hi > lo) ? (log(ora_volume(s)) - lo) / (hi - lo) : 0.0;
            double f = floor((double)nbins * t);
            if (f < 0.0) f = 0.0;
            if (f > (double)(nbins - 1)) f = (double)(nbins - 1);
            b = (int)f;
        }
    }
    if (b < 0) b = 0;
    if (b > nbins - 1) b = nbins - 1;
    return b;
}

/* Sec. 4: the distribution of blob volumes as a histogram: counts per bin and
 * the summed volume per bin (volume from the stored sigma). */
void ora_hist(int n, const float* sigma_f32, const int32_t* level, const double* sig_ladder,
              int K, int geom, int nbins, int mode, uint32_t* counts, double* vol) {
    int nb = (mode == ORA_HIST_LADDER) ? K - 1 : nbins;
    for (int b = 0; b < nb; ++b) { counts[b] = 0; if (vol) vol[b] = 0.0; }
    for (int i = 0; i < n; ++i) {
        int b = ora_bin(sigma_f32[i], level[i], sig_ladder, K, geom, nbins, mode);
        counts[b] += 1;
        if (vol) vol[b] += ora_volume((double)sigma_f32[i]);
    }
}

/* ---- Soft blob-volume histogram and its gradient (differentiable form) ----
 * Not in the paper: a smooth relaxation of the histogram used to tune the
 * sigma ladder.  Over the hard 3x3x3 local maxima of D (no threshold):
 *   H_b = sum_v sigmoid((D_v - thr) / T) * kappa_b(t(sigma_l(v))),
 * t(sigma) = (ln sigma - ln sref0) / (ln srefP - ln sref0) the normalised log
 * volume against the fixed reference ladder ends, kappa_b a triangular
 * weight of width one bin around bin centre (b + 0.5) / nbins after clamping
 * t to [0.5/nbins, 1 - 0.5/nbins] (so the weights of a blob sum to one). */
static double ora_t_of_sigma(double s, double sref0, double srefP) {
    return (log(s) - log(sref0)) / (log(srefP) - log(sref0));
}

static void ora_kappa(double t, int nbins, double* k, double* dk) {
    double lo = 0.5 / (double)nbins, hi = 1.0 - 0.5 / (double)nbins;
    int clamped = 0;
    if (t < lo) { t = lo; clamped = 1; }
    if (t > hi) { t = hi; clamped = 1; }
    for (int b = 0; b < nbins; ++b) {
        double u = (double)nbins * t - ((double)b + 0.5);
        double a = fabs(u);
        k[b] = a < 1.0 ? 1.0 - a : 0.0;
        if (dk) dk[b] = (a < 1.0 && !clamped) ? -(double)nbins * (u > 0 ? 1.0 : (u < 0 ? -1.0 : 0.0)) : 0.0;
    }
}

static double ora_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Hard local-maximum mask of D without threshold, as bytes (P x h x w). */
void ora_max_mask(const double* D, int P, int h, int w, uint8_t* mask) {
    size_t plane = (size_t)h * (size_t)w;
    for (int l = 0; l < P; ++l)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double d = D[plane * (size_t)l + (size_t)y * w + x];
                int is_max = 1;
                for (int dl = -1; dl <= 1 && is_max; ++dl)
                    for (int dy = -1; dy <= 1 && is_max; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int ll = l + dl, yy = y + dy, xx = x + dx;
                            if (ll < 0 || ll >= P || yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                            if (D[plane * (size_t)ll + (size_t)yy * w + xx] > d) { is_max = 0; break; }
                        }
                mask[plane * (size_t)l + (size_t)y * w + x] = (uint8_t)is_max;
            }
}

/* Soft histogram H[nbins].  mask may be NULL (computed from D) or a frozen
 * (K-1) x h x w byte mask. */
void ora_soft_hist(const double* img, int h, int w, const double* sig, const int* radii, int K,
                   int norm, double thr, double T, int nbins, double sref0, double srefP,
                   const uint8_t* mask_in, double* H) {
    int P = K - 1;
    size_t plane = (size_t)h * (size_t)w;
    double* D = (double*)malloc(sizeof(double) * plane * (size_t)P);
    ora_dog(img, h, w, sig, radii, K, norm, D);
    uint8_t* mask = (uint8_t*)mask_in;
    if (!mask) {
        mask = (uint8_t*)malloc(plane * (size_t)P);
        ora_max_mask(D, P, h, w, mask);
    }
    double* k = (double*)malloc(sizeof(double) * (size_t)nbins);
    for (int b = 0; b < nbins; ++b) H[b] = 0.0;
    for (int l = 0; l < P; ++l) {
        ora_kappa(ora_t_of_sigma(sig[l], sref0, srefP), nbins, k, NULL);
        for (size_t p = 0; p < plane; ++p) {
            if (!mask[plane * (size_t)l + p]) continue;
            double s = ora_sigmoid((D[plane * (size_t)l + p] - thr) / T);
            for (int b = 0; b < nbins; ++b) H[b] += s * k[b];
        }
    }
    free(k);
    if (!mask_in) free(mask);
    free(D);
}

/* Gradient of a scalar loss through the soft histogram, given gH = dloss/dH.
 * Chain rule with the mask frozen and the radii fixed:
 *   G_v = dloss/dD_v = sum_b gH_b kappa_b s (1 - s) / T,
 *   A_i = dloss/dL_i = c_i G_i - c_{i-1} G_{i-1},
 *   grad_img = sum_i blur_i^T A_i,
 *   grad_sig_i = <A_i, (dw_i (x) w_i + w_i (x) dw_i) * I>      (kernel shape)
 *              + dloss/dc_i dc_i/dsigma_i + dloss/dc_{i-1} dc_{i-1}/dsigma_i
 *              + sum_{v at level i} s sum_b gH_b dkappa_b/dt * dt/dsigma_i.
 * grad_img (h x w) and grad_sig (K) are overwritten. */
void ora_soft_grad(const double* img, int h, int w, const double* sig, const int* radii, int K,
                   int norm, double thr, double T, int nbins, double sref0, double srefP,
                   const uint8_t* mask_in, const double* gH, double* grad_img, double* grad_sig) {
    int P = K - 1;
    size_t plane = (size_t)h * (size_t)w;
    double* L = (double*)malloc(sizeof(double) * plane * (size_t)K);
    for (int i = 0; i < K; ++i) ora_blur(img, h, w, sig[i], radii[i], L + plane * (size_t)i);
    double* c = (double*)malloc(sizeof(double) * (size_t)K);
    ora_norm_coeffs(sig, K, norm, c);
    double* D = (double*)malloc(sizeof(double) * plane * (size_t)(P > 0 ? P : 1));
    for (int l = 0; l < P; ++l)
        for (size_t p = 0; p < plane; ++p)
            D[plane * (size_t)l + p] = c[l] * (L[plane * (size_t)l + p] - L[plane * (size_t)(l + 1) + p]);
    uint8_t* mask = (uint8_t*)mask_in;
    if (!mask) {
        mask = (uint8_t*)malloc(plane * (size_t)(P > 0 ? P : 1));
        ora_max_mask(D, P, h, w, mask);
    }
    double* G = (double*)calloc(plane * (size_t)(P > 0 ? P : 1), sizeof(double));
    double* k = (double*)malloc(sizeof(double) * (size_t)nbins);
    double* dk = (double*)malloc(sizeof(double) * (size_t)nbins);
    double* dloss_dc = (double*)calloc((size_t)K, sizeof(double));
    double* dloss_dt = (double*)calloc((size_t)K, sizeof(double));
    for (int l = 0; l < P; ++l) {
        ora_kappa(ora_t_of_sigma(sig[l], sref0, srefP), nbins, k, dk);
        double gk = 0.0, gdk = 0.0;
        for (int b = 0; b < nbins; ++b) { gk += gH[b] * k[b]; gdk += gH[b] * dk[b]; }
        for (size_t p = 0; p < plane; ++p) {
            if (!mask[plane * (size_t)l + p]) continue;
            double d = D[plane * (size_t)l + p];
            double s = ora_sigmoid((d - thr) / T);
            double g = gk * s * (1.0 - s) / T;
            G[plane * (size_t)l + p] = g;
            dloss_dc[l] += g * (L[plane * (size_t)l + p] - L[plane * (size_t)(l + 1) + p]);
            dloss_dt[l] += s * gdk;
        }
    }
    for (size_t p = 0; p < plane; ++p) grad_img[p] = 0.0;
    double* A = (double*)malloc(sizeof(double) * plane);
    double* Ti = (double*)malloc(sizeof(double) * plane);
    double* Tj = (double*)malloc(sizeof(double) * plane);
    for (int i = 0; i < K; ++i) {
        for (size_t p = 0; p < plane; ++p) {
            double a = 0.0;
            if (i < P) a += c[i] * G[plane * (size_t)i + p];
            if (i > 0) a -= c[i - 1] * G[plane * (size_t)(i - 1) + p];
            A[p] = a;
        }
        int r = radii[i];
        double* wk = (double*)malloc(sizeof(double) * (size_t)(2 * r + 1));
        double* dwk = (double*)malloc(sizeof(double) * (size_t)(2 * r + 1));
        ora_gauss_kernel(sig[i], r, wk);
        ora_gauss_kernel_dsigma(sig[i], r, dwk);
        ora_blur2_adjoint(A, h, w, wk, wk, r, grad_img);
        ora_blur2(img, h, w, dwk, wk, r, Ti);
        ora_blur2(img, h, w, wk, dwk, r, Tj);
        double gs = 0.0;
        for (size_t p = 0; p < plane; ++p) gs += A[p] * (Ti[p] + Tj[p]);
        grad_sig[i] = gs;
        free(dwk);
        free(wk);
    }
    /* normalisation coefficients */
    for (int l = 0; l < P; ++l) {
        if (norm == ORA_NORM_PAPER) {
            grad_sig[l] += dloss_dc[l];
        } else {
            double den = sig[l + 1] - sig[l];
            grad_sig[l] += dloss_dc[l] * sig[l + 1] / (den * den);
            grad_sig[l + 1] += -dloss_dc[l] * sig[l] / (den * den);
        }
    }
    /* bin position of each plane */
    double scale = log(srefP) - log(sref0);
    for (int l = 0; l < P; ++l) grad_sig[l] += dloss_dt[l] / (sig[l] * scale);
    free(Tj);
    free(Ti);
    free(A);
    free(dloss_dt);
    free(dloss_dc);
    free(dk);
    free(k);
    free(G);
    if (!mask_in) free(mask);
    free(D);
    free(c);
    free(L);
}

/* ------------------------------------------------------------------------
 * Preprocessing (Sec. 4, the optional first step; Table 2 times it): the
 * frame is contrast stretched to [0, 1] with a saturation fraction `sat`
 * (0.35% in the paper).  Reading: the saturation is split evenly between the
 * two ends, so with the n counts sorted ascending, c_(0) <= ... <= c_(n-1),
 * and k = floor(sat / 2 * n), the count c_(k) maps to 0, c_(n-1-k) maps to 1,
 * and values outside are clipped.  Counts are 12-bit camera values; anything
 * above 4095 is taken as 4095.  A frame whose two limits coincide maps to 0
 * at or below the limit and 1 above it. */
static int ora_int_cmp(const void* pa, const void* pb) {
    const int a = *(const int*)pa, b = *(const int*)pb;
    return (a > b) - (a < b);
}

long ora_stretch_rank(long n, double sat) { return (long)floor(sat * 0.5 * (double)n); }

int ora_stretch_limits(const uint16_t* c, long n, double sat, int32_t* lo, int32_t* hi) {
    if (n < 1) return -1;
    int* v = (int*)malloc(sizeof(int) * (size_t)n);
    if (!v) return -2;
    for (long i = 0; i < n; ++i) v[i] = c[i] > 4095 ? 4095 : (int)c[i];
    qsort(v, (size_t)n, sizeof(int), ora_int_cmp);
    long k = ora_stretch_rank(n, sat);
    if (k > (n - 1) / 2) k = (n - 1) / 2;
    *lo = v[k];
    *hi = v[n - 1 - k];
    free(v);
    return 0;
}

void ora_stretch(const uint16_t* c, long n, int32_t lo, int32_t hi, float* out) {
    for (long i = 0; i < n; ++i) {
        const int v = c[i] > 4095 ? 4095 : (int)c[i];
        double t;
        if (hi > lo) {
            t = (double)(v - lo) / (double)(hi - lo);
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
        } else {
            t = v > lo ? 1.0 : 0.0;
        }
        out[i] = (float)t;
    }
}

/* ------------------------------------------------------------------------
 * Synthetic sphere frames (Sec. 5 evaluates on frames of 100 rendered spheres
 * with Poisson and Gaussian noise; the paper names no shading model).
 * Reading: each sphere is an optically thin fluorescent droplet, so a
 * pixel's brightness is proportional to the chord length through the sphere
 * along the viewing axis, sqrt(1 - d^2 / R^2) at distance d from the centre,
 * averaged over ss x ss sub-pixel samples; the frame is a background plus the
 * spheres' contributions in table order, all in IEEE single precision with
 * the operations in the order written.  Counts are
 *   floor(lambda + sqrt(lambda) z1 + read_noise z2 + 1/2) clipped to [0, 4095],
 *   lambda = gain * intensity
 * (shot noise as a Gaussian of variance lambda, the large-count form of the
 * Poisson law, plus Gaussian read noise), in double.  z1 and z2 are sums of
 * twelve uniforms minus 6, the uniforms being the top 24 bits of Philox4x32-10
 * outputs (Salmon et al., SC'11) with counter (pixel index low, high, draw, 0)
 * and key (seed low, high): three blocks per normal. */
static void ora_mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        ora_mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        ora_mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double ora_normal12(uint64_t pix, uint32_t draw0, const uint32_t key[2]) {
    double s = 0.0;
    for (uint32_t b = 0; b < 3; ++b) {
        const uint32_t ctr[4] = {(uint32_t)pix, (uint32_t)(pix >> 32), draw0 + b, 0u};
        uint32_t r[4];
        ora_philox4x32_10(ctr, key, r);
        for (int q = 0; q < 4; ++q) s += (double)(r[q] >> 8) * (1.0 / 16777216.0);
    }
    return s - 6.0;
}

/* spheres: S x 4 floats (cx, cy, R, A); intensity (H x W float, may be NULL),
 * counts (H x W uint16).  ss in {1, 2, 4, 8}. */
int ora_render_spheres(const float* spheres, int S, int H, int W, int ss, float background, double gain,
                       double read_noise, uint64_t seed, float* intensity, uint16_t* counts) {
    if (S < 0 || H < 1 || W < 1 || !(ss == 1 || ss == 2 || ss == 4 || ss == 8)) return -1;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const float inv_n = 1.0f / (float)(ss * ss);
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            float I = background;
            for (int s = 0; s < S; ++s) {
                const float cx = spheres[4 * s], cy = spheres[4 * s + 1], R = spheres[4 * s + 2];
                const float A = spheres[4 * s + 3];
                const float inv_r2 = 1.0f / (R * R);
                float acc = 0.0f;
                for (int j = 0; j < ss; ++j) {
                    const float v = (float)y + ((float)(2 * j + 1) / (float)(2 * ss) - 0.5f);
                    const float dy = v - cy;
                    for (int i = 0; i < ss; ++i) {
                        const float u = (float)x + ((float)(2 * i + 1) / (float)(2 * ss) - 0.5f);
                        const float dx = u - cx;
                        const float q = 1.0f - (dx * dx + dy * dy) * inv_r2;
                        if (q > 0.0f) acc = acc + sqrtf(q);
                    }
                }
                I = I + A * (acc * inv_n);
            }
            if (intensity) intensity[(size_t)y * W + x] = I;
            const uint64_t pix = (uint64_t)y * (uint64_t)W + (uint64_t)x;
            const double lam = gain * (double)I;
            const double z1 = ora_normal12(pix, 0u, key), z2 = ora_normal12(pix, 3u, key);
            double n = floor(lam + sqrt(lam > 0.0 ? lam : 0.0) * z1 + read_noise * z2 + 0.5);
            if (n < 0.0) n = 0.0;
            if (n > 4095.0) n = 4095.0;
            counts[(size_t)y * W + x] = (uint16_t)n;
        }
    }
    return 0;
}
