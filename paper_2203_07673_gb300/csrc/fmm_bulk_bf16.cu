// bfloat16-input instantiations of the bulk-staged forward-role row passes.
#include "fmm_bulk.cuh"

namespace fmm {
cudaError_t launch_bulk_bf16(int mode, int vpl_mult, int depth, int mb, const PassArgs &a,
                           cudaStream_t st)
{
    return launch_bulk_typed<bf16_t>(mode, vpl_mult, depth, mb, a, st);
}
}  // namespace fmm
