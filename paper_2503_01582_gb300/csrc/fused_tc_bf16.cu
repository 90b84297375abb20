// Mixed-precision fused kernels with BF16 MLP operands (all widths and encoding sizes).
#include "split_tc.cuh"

namespace prenom {

cudaError_t launch_fused_tc_bf16(const WorkItem &one, const WorkList &wl, int W, int IN, int grid, cudaStream_t st)
{
    return launch_tc_prec<true>(one, wl, W, IN, grid, st);
}

int fused_tc_occupancy_bf16(int W, int IN, int H, bool split)
{
    return tc_occupancy_prec<true>(W, IN, H, split);
}

cudaError_t launch_sample_encode_bf16(const WorkItem &one, const WorkList &wl, int per_sm, int grid, cudaStream_t st)
{
    return launch_sample_encode_t<1>(one, wl, per_sm, grid, st);
}

}  // namespace prenom
