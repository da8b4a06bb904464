// Internal declarations of the sm_103a DoG detector (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dog.h"

namespace dogk {

// ---- fused strip kernel geometry --------------------------------------------
// A CTA owns a strip of TX output columns and walks down a band of rows in
// blocks of MB rows.  Producer warps each own a fixed set of scale levels and
// run the blur passes; NCONS consumer warps form the DoG and run the maximum
// test one block behind.  The kernel comes in two forms: 12 producer warps at
// 128 registers per thread, or 8 at 168 (both with the 4 consumer warps).
// Which is faster depends on the ladder (the host picks one, the autotuner
// times both); 10, 14 or 16 producer warps were slower than 12 on the
// 25-level ladder (level balance, spills).
constexpr int TX = 32;
constexpr int MB = 8;
constexpr int NWARPS = 12;                      // producer warps of the larger form (table sizes)
constexpr int NCONS = 4;                        // consumer (DoG + test) warps, two rows each
constexpr int RING_STRIDE = 32;    // floats per ring row (bank swizzle on row parity)
constexpr int DSLOTS = 2 * MB + 2; // DoG-buffer rows: two blocks + 2 rows of history
constexpr int MAX_LEVELS = DOG_MAX_LEVELS;
static_assert(MB % NCONS == 0, "each consumer warp tests whole rows of a block");
static_assert((NWARPS + NCONS) * 32 <= 1024, "one CTA");

// Internal pixel type: 12-bit counts contrast stretched with per-frame limits
// (the public types are DOG_DTYPE_F32 and DOG_DTYPE_U16).
constexpr int DTYPE_U16_STRETCH = 2;
constexpr int STRETCH_BINS = 4096;   // histogram bins of the 12-bit counts

enum FusedMode : int {
    MODE_CANDIDATES = 0,  // thresholded maxima -> blob list (+ pending strip-edge list)
    MODE_DUMP = 1,        // write D for every voxel
    MODE_SOFT = 2,        // soft histogram over all local maxima
    MODE_BWD = 3,         // backward prologue: dloss/dL planes and sigma partials
};

struct LevelInfo {
    int r;          // kernel radius
    int tpad;       // taps rounded up to a multiple of 8: 8 ceil((2r+1)/8)
    int e;          // chunks of MB rows the ring runs ahead: tpad / 8
    int delta;      // MB*e - r: input-row lead of this level's horizontal pass
    int ring_off;   // float offset of the ring in dynamic shared memory
    int ring_rows;  // tpad + 8 (circular, used in blocks of 8 rows)
    int woff;       // offset of this level's zero-padded full kernel (tpad floats), vertical pass
    int hoff;       // offset of the horizontal pass's copy of the same taps
};

// Candidate found at a strip edge whose 3x3x3 neighbourhood crosses into the
// neighbouring strip; settled by the resolve kernel.
struct Pending {
    int32_t frame, x, y, level;
    float response;
};

// Work unit of the persistent batched kernel.
struct FrameDesc {
    const void* img;
    int32_t h, w, pitch, dtype;
    int64_t blob_off;
    int32_t n_strips, n_bands;
    int32_t band, pad_;   // rows per band
    int64_t tile_begin;   // prefix sum of n_strips * n_bands over earlier frames
};

struct FusedParams {
    // single-frame mode (batched mode reads FrameDesc instead)
    const void* img;
    int dtype, H, W, pitch;
    const int* lohi;       // contrast-stretch limits (lo, hi) per frame (DTYPE_U16_STRETCH frames)
    int band;              // output rows per CTA (multiple of MB)
    int n_strips, n_bands;
    int overlap;           // single frame: strips of TX columns step by TX - 2 from column -1, and
                           // only lanes 1 .. TX-2 own their voxels (no strip-edge queue)
    // batched mode
    const FrameDesc* frames;
    int n_frames;
    long long n_tiles;
    const long long* ntiles_dev;  // batched: tile total written by the prep kernel
    int* tile_counter;     // persistent work counter (reset by the last CTA)
    int* done_counter;
    // ladder
    int K, P, R;
    const float* w;        // packed half kernels
    const float* c;        // P normalisation coefficients
    float thr;
    int mode;
    // outputs
    dog_blob* blobs;
    int cap;
    int* count;            // single frame: one counter; batched: per frame
    Pending* pend;
    int pend_cap;
    int* pend_count;
    float* dump;
    // soft / backward
    const float* kappa;    // P x nbins triangular weights per plane
    const float* dkappa;   // P x nbins derivative wrt t
    const float* gH;       // nbins dloss/dH
    int nbins;
    float inv_T;
    float* soft_out;       // nbins (global, float accumulation)
    float* A;              // K x H x W dloss/dL planes (MODE_BWD)
    double* dc_acc;        // P: dloss/dc
    double* dt_acc;        // P: dloss/dt
    dog_soft_max* rec;     // MODE_SOFT: maxima recorded for the backward (or nullptr)
    int rec_cap;
    int* rec_count;
    int* status;
    // shared-memory layout (floats)
    int in_off, in_rows, in_stride;
    int d_off;
    int w_off, w_total;
    int dmin, dmax;
    int smem_bytes;
    int nw;                // producer warps of the kernel form (8 or 12)
    int warp_nlev[NWARPS];
    unsigned char warp_lev[NWARPS][MAX_LEVELS];
    LevelInfo lv[MAX_LEVELS];
};

struct ResolveParams {
    const Pending* pend;
    const int* pend_count;
    int pend_cap;
    const FrameDesc* frames;  // batched: per-frame image; single: frames == nullptr
    const void* img;
    int dtype, H, W, pitch;
    const int* lohi;          // contrast-stretch limits per frame (as FusedParams)
    int K, P;
    const float* w;
    const float* c;
    int woff[MAX_LEVELS];
    int r[MAX_LEVELS];
    dog_blob* blobs;
    int cap;
    int* count;
    int* status;
};

// ---- launchers (defined in the .cu files) -----------------------------------
cudaError_t launch_fused(const FusedParams& p, int grid, cudaStream_t s);
cudaError_t launch_resolve(const ResolveParams& p, int max_pending, cudaStream_t s);
cudaError_t launch_batch_prep(const dog_frame* frames, int n, int band, int tail_tiles, int blob_cap,
                              bool stretch, FrameDesc* desc, long long* cand_off, long long* out_off, int* hw,
                              long long* ntiles, cudaStream_t s);
// contrast stretch (dog_stretch.cu): per-frame histograms (STRETCH_BINS ints
// per frame, zeroed here) and limits lohi (2 ints per frame) of the single
// frame (frames == nullptr) or of the U16 frames of a device frame table
cudaError_t launch_stretch_limits(const dog_frame* frames, int n, const uint16_t* img, int H, int W, int pitch,
                                  double sat, int num_sms, int* hist, int* lohi, cudaStream_t s);
// FFT-convolution backend (dog_fft.cu)
struct FftWS;
int fft_create(FftWS** out, int max_h, int max_w, int K, int R, const std::vector<std::vector<double>>& w);
void fft_free(FftWS* f);
int fft_run(FftWS* f, const void* img, int dtype, int H, int W, int pitch, const int* lohi, int P,
            const float* c, float thr, int mode, dog_blob* blobs, int cap, int* count, float* dump, int* status,
            cudaStream_t s);
cudaError_t launch_stretch_apply(const uint16_t* img, int H, int W, int pitch, const int* lohi, float* out,
                                 int out_pitch, int num_sms, cudaStream_t s);

struct HistParams {
    const dog_blob* blobs;
    const int* count;        // per frame
    int cap;
    const long long* off;    // per frame offset (nullptr: 0)
    int n_frames;
    int P, nbins, mode;      // mode: DOG_HIST_LOGV / DOG_HIST_LADDER
    const float* sig_f;      // P plane sigmas rounded to float (on-ladder test)
    const int* level_bin;    // P: bin of an on-ladder blob
    const double* log_sig;   // P: ln sigma of each plane (double)
    double log_lo, log_hi;   // ln sigma of the first / last DoG plane
    unsigned* hist;          // n_frames x nbins_out
    double* vol;             // n_frames x nbins_out or nullptr
};
cudaError_t launch_hist(const HistParams& p, cudaStream_t s);

struct PruneParams {
    const dog_blob* cand;
    const int* cand_count;   // per frame
    int cap_in;
    const long long* cand_off;  // per-frame offset of candidates (nullptr: 0)
    int n_frames;
    const int* frame_hw;     // 2 ints per frame (h, w) or nullptr (use H, W)
    int H, W;
    int P;
    const double* sig;       // P plane sigmas (double)
    const int* d2thr;        // P x P: squared distance below which two planes' discs conflict
    int cell;                // grid cell edge (pixels)
    int mode;
    int* state;              // scratch: per candidate
    int* target;             // scratch: per candidate
    int* order;              // scratch: per candidate
    dog_blob* out;
    int cap_out;
    const long long* out_off;  // per frame output offset (nullptr: 0)
    int* out_count;          // per frame
    int* status;
    int max_rounds;
    // optional: the volume histogram of each frame's pruned blobs, computed by
    // the same CTA after compaction (hist.hist non-null; hist.off, .blobs,
    // .count and .cap are not used: the kernel's own output is binned)
    HistParams hist;
};
cudaError_t launch_prune(const PruneParams& p, cudaStream_t s);


}  // namespace dogk
