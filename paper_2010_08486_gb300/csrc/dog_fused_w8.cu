// Fused DoG detector kernel: the 8-producer-warp forms (dog_fused_forms.cuh),
// compiled apart from the 12-warp ones so the two build in parallel.
#include "dog_fused_forms.cuh"

namespace dogk {

cudaError_t launch_fused_w8(const FusedParams& p, int grid, cudaStream_t s) { return launch_fused_form<8>(p, grid, s); }

}  // namespace dogk
