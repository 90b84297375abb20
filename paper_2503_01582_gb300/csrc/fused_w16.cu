// Fused FP32 kernels for MLP width 16 (all encoding widths and tile sizes).
#include "fused_fp32_kernel.cuh"

namespace prenom {

cudaError_t launch_fused_fp32_w16(const WorkItem &one, const WorkList &wl, int IN, int S, int grid, cudaStream_t st)
{
    return launch_fused_w<16>(one, wl, IN, S, grid, st);
}

}  // namespace prenom
