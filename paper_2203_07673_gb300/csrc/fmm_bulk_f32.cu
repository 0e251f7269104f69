// float32 instantiations of the bulk-staged forward-role row passes.
#include "fmm_bulk.cuh"

namespace fmm {
cudaError_t launch_bulk_f32(int mode, int vpl_mult, int depth, int mb, const PassArgs &a,
                           cudaStream_t st)
{
    return launch_bulk_typed<float>(mode, vpl_mult, depth, mb, a, st);
}
}  // namespace fmm
