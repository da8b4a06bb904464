/*
 * dog.h - C ABI of the GB300 (sm_103a) Difference-of-Gaussians blob detector.
 *
 * Method: arXiv 2010.08486, "Towards Online Steering of Flame Spray Pyrolysis
 * Nanoparticle Synthesis".  Sec. 3 defines the scale space L = g(sigma) * I;
 * Sec. 4 the sigma ladder (Eq. 1), adjacent differences (Eq. 2), the scale
 * normalisation (Eq. 3), the maximum-filter extremum test, pruning by overlap
 * and the blob-volume histogram; Sec. 4.1 the 3x3x3 maximum pooling, the
 * threshold Thresh = (MaxPool3D(D) - D == 0) and (D > 0.1), and coalescing of
 * blobs whose normalised overlap exceeds 0.5.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* are CUDA device pointers owned by the caller; h_*
 *    are host pointers.  The library never frees caller memory.
 *  - Images are row-major, one channel, pitch counted in ELEMENTS (>= w).
 *    dtype DOG_DTYPE_F32: float in any range (the paper's frames are in
 *    [0, 1]).  DOG_DTYPE_U16: 12-bit counts, converted on load to
 *    float(v) / 4095 (one IEEE single division).
 *  - Coordinates: x = column, y = row, integer pixel centres.  `level` is the
 *    DoG plane index i (0 .. K-2) whose sigma is sigma_i (the smaller sigma
 *    of the pair, Eq. 3).
 *  - The boundary is half-sample symmetric reflection (... 1 0 | 0 1 2 ...),
 *    folded repeatedly when a kernel radius exceeds the frame.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Every compute
 *    call is asynchronous and stream-ordered; it returns DOG_OK once the work
 *    is enqueued.  Errors found later on the device (capacity overflow, a
 *    wait that ran out) are recorded in the handle's status word, read with
 *    dog_get_status.
 *  - A handle owns device workspace that its calls reuse: calls on one handle
 *    must be ordered on one stream (or otherwise serialised).  Use one handle
 *    per concurrent stream or host thread.
 *  - No call throws, traps or aborts; all return a dog_status code.
 */
#ifndef DOG_H_
#define DOG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum dog_status {
    DOG_OK = 0,
    DOG_ERR_INVALID = -1,     /* bad argument (null pointer, size, config)       */
    DOG_ERR_NOMEM = -2,       /* device or host allocation failed                */
    DOG_ERR_CUDA = -3,        /* a CUDA runtime call failed                      */
    DOG_ERR_CAPACITY = -4,    /* a blob list overflowed (true count still given) */
    DOG_ERR_TIMEOUT = -5,     /* a bounded device wait ran out                   */
    DOG_ERR_UNSUPPORTED = -6  /* valid but outside what this build supports      */
} dog_status;

enum { DOG_LADDER_GEOM = 0, DOG_LADDER_ARITH = 1 };
enum { DOG_NORM_DERIV = 0, DOG_NORM_PAPER = 1 };
enum { DOG_PRUNE_COALESCE = 0, DOG_PRUNE_SUPPRESS = 1, DOG_PRUNE_OFF = 2 };
enum { DOG_HIST_LOGV = 0, DOG_HIST_LADDER = 1 };
enum { DOG_DTYPE_F32 = 0, DOG_DTYPE_U16 = 1 };
enum { DOG_BACKEND_DIRECT = 0, DOG_BACKEND_FFT = 1 };

/* Largest ladder and radius this build accepts. */
#define DOG_MAX_LEVELS 32
#define DOG_MAX_RADIUS 64
#define DOG_MAX_NBINS 256

/* ---------------------------------------------------------------- config
 * Hyper-parameters of Sec. 4 / 4.1 (n_bin = n_levels - 1, min_sigma,
 * max_sigma, truncate, threshold, overlap) plus the readings this library
 * takes where the paper is silent.
 *
 *  n_levels   Gaussian levels K (K-1 DoG planes).  0: for GEOM, derived from
 *             max_sigma as K = floor(ln(max/min)/ln(ratio)) + 2, so the DoG
 *             planes span [min_sigma, max_sigma].  Required for ARITH.
 *  sigmas     optional explicit ladder (host pointer, n_levels increasing
 *             values); copied by dog_create.  NULL: use `ladder`.
 *  ladder     GEOM: sigma_i = min_sigma * ratio^i.  ARITH: Eq. 1,
 *             sigma_i = min + i (max - min) / (K - 1).
 *  truncate   kernel radius r_i = floor(truncate * sigma_i + 0.5) (Sec. 4.1).
 *  threshold  strict lower bound on the response D (Sec. 4.1, default 0.1).
 *  overlap    normalised disc overlap above which blobs coalesce (0.5).
 *  norm       DERIV: c_i = sigma_i / (sigma_{i+1} - sigma_i), the finite-
 *             difference form of sigma * dg/dsigma (Sec. 3).  PAPER: c_i =
 *             sigma_i (Eq. 3 literally).  D_i = c_i (L_i - L_{i+1}).
 *  prune      COALESCE (mean sigma of the group), SUPPRESS, or OFF.
 *  nbins      LOGV bins on log volume between the first and last DoG plane;
 *             LADDER uses one bin per DoG plane (nbins ignored).
 *  soft_T     temperature of the soft (sigmoid) threshold, differentiable form.
 *  max_h/max_w  largest frame a call will pass (sizes workspace).
 *  blob_cap   candidate capacity per frame held in the workspace.
 *  stretch_sat  contrast stretch of 12-bit frames (Sec. 4, the optional
 *             preprocessing step; the paper uses 0.0035): 0 = off.  When set,
 *             every DOG_DTYPE_U16 frame a detection call ingests is mapped to
 *             [0, 1] with its own limits as in dog_stretch_limits/dog_stretch
 *             (computed on the device before the detection kernel, applied as
 *             the kernel loads the counts); FP32 frames are used as given.
 *  backend    DIRECT: the fused separable passes (default).  FFT: the scale
 *             space by FFT convolution (Sec. 4.1's alternative): the frame,
 *             reflect-padded by the largest radius, is transformed once and
 *             each level is the inverse transform of its product with the
 *             level's kernel spectrum (single precision), then the same DoG,
 *             3x3x3 test and threshold.  Used by dog_candidates, dog_detect
 *             and dog_debug_dog; dog_detect_batched returns UNSUPPORTED and the
 *             differentiable form always uses the direct passes.  Its
 *             workspace (about 10 K max_h max_w bytes) is allocated by the
 *             first such call.  An FFT handle may hold a ladder whose direct
 *             passes would not fit in shared memory; its differentiable calls
 *             then return UNSUPPORTED.
 */
typedef struct dog_config {
    int32_t n_levels;
    const double* sigmas;
    double min_sigma, max_sigma, ratio;
    int32_t ladder;
    double truncate, threshold, overlap;
    int32_t norm, prune;
    int32_t nbins, hist_mode;
    double soft_T;
    int32_t max_h, max_w;
    int32_t blob_cap;
    double stretch_sat;
    int32_t backend;
} dog_config;

/* One blob: centre (x, y), DoG plane, sigma (the plane's sigma, or the mean
 * sigma of a coalesced group), response D at the centre.  20 bytes.
 * Radius r = sqrt(2) sigma, volume V = 4/3 pi r^3 (Sec. 4). */
typedef struct dog_blob {
    int32_t x, y, level;
    float sigma, response;
} dog_blob;

/* One frame of a batched call (the table lives in DEVICE memory).
 * blob_off: first slot of this frame's blobs in the output array; each frame
 * owns blob_cap slots (dog_config.blob_cap). */
typedef struct dog_frame {
    const void* ptr;
    int32_t h, w, pitch, dtype;
    int64_t blob_off;
} dog_frame;

typedef struct dog_handle dog_t;

/* Fill *cfg with the defaults: GEOM ladder 1.0 .. 10.0 ratio 1.6, truncate
 * 4, threshold 0.1, overlap 0.5, DERIV, COALESCE, 32 LOGV bins, soft_T 0.01,
 * max frame 1024x1024, blob_cap 65536, no contrast stretch. */
int dog_config_default(dog_config* cfg);

/* Build a detector on the current CUDA device: computes the ladder, radii,
 * kernels (double, rounded to float) and normalisation on the host, uploads
 * them, and allocates the workspace.  *out receives the handle (NULL on
 * failure).  Errors: INVALID (config), UNSUPPORTED (K > DOG_MAX_LEVELS,
 * radius > DOG_MAX_RADIUS, or shared memory needs above the device limit),
 * NOMEM, CUDA. */
int dog_create(const dog_config* cfg, dog_t** out);

/* Release the handle and its workspace (synchronises the device).  NULL ok. */
void dog_destroy(dog_t* h);

/* Introspection (host): K, the ladder sigma_0..K-1, radii, normalisation
 * c_0..K-2.  Any output pointer may be NULL. */
int dog_ladder(const dog_t* h, int32_t* K, double* h_sigmas, int32_t* h_radii, double* h_norm);

/* Candidates only (Sec. 4.1 Thresh): every voxel with D > threshold that no
 * in-range 3x3x3 neighbour exceeds.  Writes up to `cap` blobs to d_blobs (in
 * no particular order) and the TRUE count to *d_count (may exceed cap: the
 * status word then records DOG_ERR_CAPACITY).  One fused pass: all scales of
 * a tile from one read of the frame; D is never stored. */
int dog_candidates(dog_t* h, const void* d_img, int32_t dtype, int32_t img_h, int32_t img_w,
                   int32_t pitch, dog_blob* d_blobs, int32_t cap, int32_t* d_count, void* stream);

/* Overlap pruning of Sec. 4.1 on a candidate list (device): visit candidates
 * by decreasing response (ties: level, y, x); each joins the first already
 * accepted blob it overlaps by more than `overlap` (normalised disc overlap,
 * r = sqrt(2) sigma of each plane) or is accepted.  COALESCE reports the mean
 * sigma of each group (summed in visiting order; the plane sigma exactly when
 * all members share one plane), SUPPRESS drops joiners, OFF copies.  Frame
 * size (img_h, img_w) bounds the coordinates.  n = min(*d_count, cap_in).
 * Output: up to cap_out blobs, count in *d_nout. */
int dog_prune(dog_t* h, const dog_blob* d_cand, const int32_t* d_count, int32_t cap_in,
              int32_t img_h, int32_t img_w, dog_blob* d_out, int32_t cap_out, int32_t* d_nout,
              void* stream);

/* Pruning without a handle and without allocating anything.  The paper has
 * no counterpart: this is a convenience for callers that may not allocate
 * device memory themselves, such as a plug-in whose host framework owns all
 * device memory and forbids allocations inside its execution step, or a
 * real-time loop that must not stall on the allocator.  Same result as
 * dog_prune for the same candidate list.
 *
 *  h_sigmas   the n_planes DoG-plane sigmas (host, increasing), i.e. the
 *             ladder's first K-1 values; candidate levels index them.  Read
 *             on the host during the call (passed to the GPU as a kernel
 *             parameter), so the caller may reuse the array on return.
 *  overlap    threshold on the normalised disc overlap, in [0, 1).
 *  mode       DOG_PRUNE_COALESCE, DOG_PRUNE_SUPPRESS or DOG_PRUNE_OFF.
 *  d_cand, d_count, cap_in, d_out, cap_out, d_nout   as in dog_prune.
 *
 * Scratch memory is a fixed array inside the library, sized for
 * DOG_NOALLOC_MAX_CAND candidates (about 0.8 MB, held by every GPU that
 * loads the library until the process exits): cap_in above that limit
 * returns DOG_ERR_UNSUPPORTED.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the array and it keeps the last
 * call's contents (each call rewrites its tables and the per-candidate
 * state), so calls whose GPU work may overlap (other streams, other host
 * threads) race: serialise them on one stream.  There is no handle and no
 * status word to read: overflow of cap_out shows only as *d_nout > cap_out
 * (the true count), and errors of the launch itself come back as the return
 * code. */
#define DOG_NOALLOC_MAX_CAND 65536
int dog_prune_noalloc(const dog_blob* d_cand, const int32_t* d_count, int32_t cap_in,
                      const double* h_sigmas, int32_t n_planes, double overlap, int32_t mode,
                      dog_blob* d_out, int32_t cap_out, int32_t* d_nout, void* stream);

/* Contrast-stretch limits of one frame of 12-bit counts (Sec. 4: the optional
 * preprocessing step stretches a frame to [0, 1] with a saturation of 0.35%).
 * With the n = img_h * img_w counts sorted ascending (counts above 4095 count
 * as 4095) and k = floor(sat / 2 * n) (at most (n-1)/2), d_lohi[0] receives
 * the count at rank k and d_lohi[1] the count at rank n-1-k (device, two
 * int32).  d_hist is caller-owned device scratch of 4096 int32 (overwritten).
 * sat in [0, 1); frames of 2^31 pixels or more are not supported.  No
 * allocation; stream-ordered. */
int dog_stretch_limits(const uint16_t* d_img, int32_t img_h, int32_t img_w, int32_t pitch, double sat,
                       int32_t* d_hist, int32_t* d_lohi, void* stream);

/* The stretched frame: d_out[y * out_pitch + x] = clamp((c - lo) / (hi - lo),
 * 0, 1) for the count c (4095 at most) of pixel (x, y), as one IEEE single
 * division of the two exact integers; lo = d_lohi[0], hi = d_lohi[1] (device);
 * when hi == lo the result is 0 for c <= lo and 1 above.  FP32 output,
 * row-major, pitch in elements. */
int dog_stretch(const uint16_t* d_img, int32_t img_h, int32_t img_w, int32_t pitch, const int32_t* d_lohi,
                float* d_out, int32_t out_pitch, void* stream);

/* Synthetic frame of rendered spheres (Sec. 5 evaluates on 1000 x 1000
 * frames of 100 rendered spheres with Poisson and Gaussian noise; the paper
 * names no shading model, so the one below is this library's reading).
 *  d_spheres   n_spheres x 4 floats (cx, cy, R, A), device, 16-byte aligned;
 *              at most 8192 spheres.
 *  intensity   background + sum over spheres (table order) of
 *              A * mean over ss x ss sub-pixel samples of sqrt(max(0, 1 -
 *              d^2/R^2)) (chord length of an optically thin sphere), pixel
 *              centres at integer coordinates, single precision with every
 *              operation rounded as written; written to d_intensity (row
 *              pitch img_w) unless it is NULL.  ss in {1, 2, 4, 8}.
 *  counts      floor(lambda + sqrt(lambda) z1 + read_noise z2 + 1/2) clipped
 *              to [0, 4095], lambda = gain * intensity, in double; z1, z2 are
 *              sums of twelve uniforms minus 6, the uniforms being the top 24
 *              bits of Philox4x32-10 blocks with counter (y * img_w + x low
 *              and high word, draw, 0) and key (seed low, high), draws 0..2
 *              for z1 and 3..5 for z2.  uint16, row pitch `pitch` elements.
 * No allocation; stream-ordered. */
int dog_render_spheres(const float* d_spheres, int32_t n_spheres, int32_t img_h, int32_t img_w, int32_t ss,
                       float background, double gain, double read_noise, uint64_t seed, float* d_intensity,
                       uint16_t* d_counts, int32_t pitch, void* stream);

/* Blob-volume histogram (Sec. 4, Sec. 4.1: the pruned blobs are binned by volume).
 * d_hist: uint32 counts (nbins, or K-1 in LADDER mode), overwritten.
 * d_hist_vol: optional (NULL ok) double sum of V per bin, overwritten.
 * A blob whose stored sigma equals its plane's sigma (as float) is binned by
 * its plane alone; otherwise bin = floor(nbins (ln V - lo) / (hi - lo)),
 * clamped, lo/hi = ln V of the first/last DoG plane sigma. */
int dog_volume_hist(dog_t* h, const dog_blob* d_blobs, const int32_t* d_count, int32_t cap,
                    uint32_t* d_hist, double* d_hist_vol, void* stream);

/* Whole method on one frame: candidates -> prune -> histogram.  d_blobs gets
 * the pruned blobs (up to cap), *d_count their number; d_hist / d_hist_vol as
 * in dog_volume_hist (either may be NULL). */
int dog_detect(dog_t* h, const void* d_img, int32_t dtype, int32_t img_h, int32_t img_w,
               int32_t pitch, dog_blob* d_blobs, int32_t cap, int32_t* d_count, uint32_t* d_hist,
               double* d_hist_vol, void* stream);

/* Batched detection of n frames of uneven sizes (d_frames: device table).
 * One persistent launch walks all (frame, strip, row band) tiles from a work
 * counter; then one pruning and one histogram launch cover every frame.
 * Frame f's pruned blobs go to d_blobs[d_frames[f].blob_off ...] (at most
 * blob_cap), its count to d_counts[f], its histogram to
 * d_hists[f * nbins_out ...] (nbins_out = nbins, or K-1 in LADDER mode).
 * Tile shapes come from the handle's tuning (dog_set_tiling).  h_max_h and
 * h_max_w bound the frame sizes of this call (host values). */
int dog_detect_batched(dog_t* h, const dog_frame* d_frames, int32_t n, int32_t h_max_h,
                       int32_t h_max_w, dog_blob* d_blobs, int32_t* d_counts, uint32_t* d_hists,
                       void* stream);

/* Row-band height used by detection tiles (a multiple of 8, or 0 for whole
 * frames) and the persistent grid multiplier; set by the autotuner. */
int dog_set_tiling(dog_t* h, int32_t band_rows, int32_t ctas_per_sm);

/* Producer warps of the detection kernel form: 8 (168 registers each) or 12
 * (128 each), or 0 for the handle's default choice (12 for ladders of 20 or
 * more levels whose largest level fits an even share of 12 warps, else 8).
 * Results do not depend on it: every level is computed by the same
 * operations in either form.  Set by the autotuner; the scale levels are
 * re-balanced over the chosen warps on the host.  Not safe to call while a
 * launch on this handle is being issued from another thread.
 * Errors: INVALID (n not 0, 8 or 12). */
int dog_set_producer_warps(dog_t* h, int32_t n);

/* The handle's current producer-warp count (8 or 12), or INVALID for NULL. */
int dog_get_producer_warps(const dog_t* h);

/* Differentiable form (not in the paper; used to tune the ladder).  Soft
 * histogram over the hard 3x3x3 local maxima of D (no threshold):
 *   H_b += sum_v sigmoid((D_v - threshold) / soft_T) kappa_b(t(sigma_l(v)))
 * with t the normalised log volume against the handle's own ladder ends and
 * kappa_b a triangular weight one bin wide (t clamped to the bin centres).
 * d_sigmas: K float sigmas (device) replacing the ladder; radii stay fixed.
 * d_soft_hist: nbins floats, ACCUMULATED (+=) so that frames can be summed. */
int dog_soft_hist(dog_t* h, const float* d_img, int32_t img_h, int32_t img_w, int32_t pitch,
                  const float* d_sigmas, float* d_soft_hist, void* stream);

/* Backward of dog_soft_hist for dloss/dH = d_grad_hist (nbins floats).
 * Recomputes the blur levels (none are kept from the forward) and writes
 * dloss/dI to d_grad_img (img_h x img_w, row-major, pitch img_w, overwritten)
 * and ACCUMULATES dloss/dsigma into d_grad_sigmas (K floats).  The maximum
 * mask is recomputed at the given sigmas and treated as constant. */
int dog_backward(dog_t* h, const float* d_img, int32_t img_h, int32_t img_w, int32_t pitch,
                 const float* d_sigmas, const float* d_grad_hist, float* d_grad_img,
                 float* d_grad_sigmas, void* stream);

/* One hard local maximum v of the soft histogram's forward pass, as the
 * backward needs it (the mask is held constant): voxel (x, y, level l),
 * q = s_v (1 - s_v) / soft_T, qe = q (L_l - L_{l+1})(v) and s = s_v, with
 * s_v = sigmoid((D_v - threshold) / soft_T).  24 bytes. */
typedef struct dog_soft_max {
    int32_t x, y, level;
    float q, qe, s;
} dog_soft_max;

/* dog_soft_hist that also records every maximum into d_max (device, up to
 * cap entries, in no particular order); *d_count (device) receives their true
 * number, so *d_count > cap means the list is incomplete (the status word is
 * then DOG_ERR_CAPACITY and the list must not be passed to dog_backward_rec). */
int dog_soft_hist_rec(dog_t* h, const float* d_img, int32_t img_h, int32_t img_w, int32_t pitch,
                      const float* d_sigmas, float* d_soft_hist, dog_soft_max* d_max, int32_t cap,
                      int32_t* d_count, void* stream);

/* Backward of dog_soft_hist_rec from its list of maxima (same frame, same
 * d_sigmas): the dloss/dL planes are scattered from the list and no blur level
 * is recomputed; then the same adjoint blurs as dog_backward.  Outputs as in
 * dog_backward.  An incomplete list (*d_count > cap) sets DOG_ERR_CAPACITY and
 * uses the first cap entries. */
int dog_backward_rec(dog_t* h, const float* d_img, int32_t img_h, int32_t img_w, int32_t pitch,
                     const float* d_sigmas, const dog_soft_max* d_max, const int32_t* d_count, int32_t cap,
                     const float* d_grad_hist, float* d_grad_img, float* d_grad_sigmas, void* stream);

/* Debug/parity: write the DoG cube D (K-1 x img_h x img_w floats, row-major
 * planes) computed by the same fused kernel as dog_candidates. */
int dog_debug_dog(dog_t* h, const void* d_img, int32_t dtype, int32_t img_h, int32_t img_w,
                  int32_t pitch, float* d_dog, void* stream);

/* Rolling per-stream histogram for the serving loop: adds d_hist (nbins
 * uint32) into ring slot (*d_head % window) of d_ring (window x nbins),
 * subtracting the slot's previous content from the running sum d_sum (nbins
 * uint32), then advances *d_head.  All device memory, one launch. */
int dog_ring_hist_push(const uint32_t* d_hist, int32_t nbins, uint32_t* d_ring, int32_t window,
                       uint32_t* d_sum, int32_t* d_head, void* stream);

/* The same for a batch of n frames from several streams in one launch:
 * frame f's histogram d_hists[f * nbins ...] goes to stream d_stream_ids[f]
 * (0 <= id < n_streams), whose ring is d_rings[id * window * nbins ...], sum
 * d_sums[id * nbins ...] and head d_heads[id].  Frames of one stream are
 * pushed in batch order. */
int dog_ring_hist_push_batched(const uint32_t* d_hists, const int32_t* d_stream_ids, int32_t n,
                               int32_t nbins, int32_t n_streams, uint32_t* d_rings, int32_t window,
                               uint32_t* d_sums, int32_t* d_heads, void* stream);

/* Measurement.  While enabled, every launch of the fused detection kernel
 * (candidates, batched, debug and differentiable forms) is bracketed by a pair
 * of CUDA events recorded on the launch's own stream (up to 65536 launches
 * between reads; later ones are not timed).  dog_profile_read waits for the
 * recorded events, returns the summed kernel time in milliseconds and the
 * number of timed launches, and clears them. */
int dog_profile_enable(dog_t* h, int32_t enable);
int dog_profile_read(dog_t* h, double* h_ms, int32_t* h_launches);

/* Measured single-precision multiply-add peak of the current GPU, the
 * roofline denominator of the detection kernels (no counterpart in the
 * paper).  A grid of 4 CTAs x 256 threads per SM runs 16 independent FMA
 * chains per thread from registers, `iters` x 64 FMAs per thread; pair != 0
 * issues them as packed two-lane FMAs (two per instruction).  The launch is
 * timed `reps` times with CUDA events on `stream` after one short warm-up;
 * *h_tflops receives the median rate (2 flop per FMA), *h_ms (NULL ok) the
 * median launch time.  Allocates and frees 4 bytes of device memory;
 * synchronises the stream. */
int dog_fma_peak(int32_t pair, int64_t iters, int32_t reps, double* h_tflops, double* h_ms, void* stream);

/* Read and clear the handle's device status word (synchronises the stream
 * passed to the last call).  *h_status receives DOG_OK or the first error. */
int dog_get_status(dog_t* h, int32_t* h_status);

/* Testing: make the library's device workspace allocations (dog_create and
 * the growth of the batched workspace) fail on purpose.  After this call the
 * next `after` such allocations succeed and the one following them reports
 * out of memory without calling the CUDA allocator, so the caller sees
 * DOG_ERR_NOMEM and the library frees what it had allocated; later ones succeed
 * again.  -1 switches the injection off.  Process-wide; no counterpart in the
 * paper. */
int dog_test_fail_alloc(int32_t after);

/* Human-readable name of a status code (static string). */
const char* dog_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* DOG_H_ */
