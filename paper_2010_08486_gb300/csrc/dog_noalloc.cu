// Overlap pruning for callers that cannot allocate device memory.
//
// dog_prune_noalloc runs the same pruning kernel as dog_prune, but needs no
// handle and allocates nothing: its scratch memory (the per-candidate state,
// target and order arrays, the conflict table, the plane sigmas and a status
// word) lives in one file-scope device array of fixed size.  Every GPU that
// loads this library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address; on each device,
// the first call looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it.  The per-call tables (conflict distances and
// plane sigmas) are computed on the host and passed BY VALUE as a kernel
// parameter to a one-CTA set-up kernel that writes them into the array, so no
// call copies from host memory.  Calls share the array, so calls whose GPU
// work overlaps (different streams, or other host threads) race on it; order
// them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dog_internal.cuh"

namespace dogk {
int conflict_d2(double sa, double sb, double thr);
}

using namespace dogk;

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kTableBytes = sizeof(int) * MAX_LEVELS * MAX_LEVELS;   // conflict table
constexpr size_t kSigBytes = sizeof(double) * MAX_LEVELS;               // plane sigmas
constexpr size_t kStatusBytes = 256;                                     // status word (padded)
constexpr size_t kHeadBytes = kTableBytes + kSigBytes + kStatusBytes;
constexpr size_t kScratchBytes = kHeadBytes + sizeof(int) * 3 * (size_t)DOG_NOALLOC_MAX_CAND;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_lock;
void* g_addr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Per-call tables, passed by value (about 4.4 KB of kernel parameters).
struct NoallocTables {
    int d2[MAX_LEVELS * MAX_LEVELS];   // P x P conflict distances, row-major
    double sig[MAX_LEVELS];            // plane sigmas
    int P;
};

__global__ void noalloc_setup_kernel(const __grid_constant__ NoallocTables t, int* d2thr, double* sig,
                                     int* status) {
    for (int q = threadIdx.x; q < t.P * t.P; q += blockDim.x) d2thr[q] = t.d2[q];
    for (int q = threadIdx.x; q < t.P; q += blockDim.x) sig[q] = t.sig[q];
    if (threadIdx.x == 0) *status = 0;
}

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int dog_prune_noalloc(const dog_blob* d_cand, const int32_t* d_count, int32_t cap_in,
                                 const double* h_sigmas, int32_t n_planes, double overlap, int32_t mode,
                                 dog_blob* d_out, int32_t cap_out, int32_t* d_nout, void* stream) {
    if (!d_cand || !d_count || !d_out || !d_nout || !h_sigmas || cap_in < 0 || cap_out < 0) return DOG_ERR_INVALID;
    if (n_planes < 1 || n_planes > MAX_LEVELS - 1) return DOG_ERR_INVALID;
    if (!(overlap >= 0.0 && overlap < 1.0)) return DOG_ERR_INVALID;
    if (mode < DOG_PRUNE_COALESCE || mode > DOG_PRUNE_OFF) return DOG_ERR_INVALID;
    if (cap_in > DOG_NOALLOC_MAX_CAND) return DOG_ERR_UNSUPPORTED;   // beyond the fixed scratch
    for (int l = 0; l < n_planes; ++l)
        if (!(h_sigmas[l] > 0.0)) return DOG_ERR_INVALID;

    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return DOG_ERR_CUDA;
    unsigned char* b = static_cast<unsigned char*>(base);
    int* d2thr = reinterpret_cast<int*>(b);
    double* sig = reinterpret_cast<double*>(b + kTableBytes);
    int* status = reinterpret_cast<int*>(b + kTableBytes + kSigBytes);
    int* state = reinterpret_cast<int*>(b + kHeadBytes);
    int* target = state + DOG_NOALLOC_MAX_CAND;
    int* order = target + DOG_NOALLOC_MAX_CAND;

    // conflict table and cell size, on the host (same rule as dog_create)
    const int P = n_planes;
    NoallocTables t;
    int maxd2 = 1;
    for (int a = 0; a < P; ++a) {
        t.sig[a] = h_sigmas[a];
        for (int q = 0; q < P; ++q) {
            t.d2[a * P + q] = conflict_d2(h_sigmas[a], h_sigmas[q], overlap);
            if (t.d2[a * P + q] > maxd2) maxd2 = t.d2[a * P + q];
        }
    }
    t.P = P;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps the last call's contents: the tables and the status word
    // are rewritten here; the pruning kernel initialises the per-candidate state
    noalloc_setup_kernel<<<1, 256, 0, s>>>(t, d2thr, sig, status);
    if (cudaGetLastError() != cudaSuccess) return DOG_ERR_CUDA;
    PruneParams q{};
    q.cand = d_cand;
    q.cand_count = d_count;
    q.cap_in = cap_in;
    q.n_frames = 1;
    q.H = 1;
    q.W = 1;
    q.P = P;
    q.sig = sig;
    q.d2thr = d2thr;
    q.cell = (int)std::ceil(std::sqrt((double)maxd2));
    if (q.cell < 1) q.cell = 1;
    q.mode = mode;
    q.state = state;
    q.target = target;
    q.order = order;
    q.out = d_out;
    q.cap_out = cap_out;
    q.out_count = d_nout;
    q.status = status;
    return launch_prune(q, s) == cudaSuccess ? DOG_OK : DOG_ERR_CUDA;
}
