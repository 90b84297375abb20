// Mixed-precision fused kernels with FP16 MLP operands (all widths and encoding sizes).
#include "fused_tc.cuh"

namespace prenom {

cudaError_t launch_fused_tc_fp16(const ObjDesc &od, const BatchDesc &bd, int grid, cudaStream_t st)
{
    return launch_tc_prec<false>(od, bd, grid, st);
}

}  // namespace prenom
