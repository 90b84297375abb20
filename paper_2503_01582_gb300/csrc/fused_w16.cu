// Fused FP32 kernels for MLP width 16 (all encoding widths and tile sizes).
#include "fused_fp32.cuh"

namespace prenom {

cudaError_t launch_fused_fp32_w16(const ObjDesc &od, const BatchDesc &bd, int S, int grid, cudaStream_t st)
{
    return launch_fused_w<16>(od, bd, S, grid, st);
}

}  // namespace prenom
