// float32 instantiations of the staged row-pass kernels.
#include "fmm_staged.cuh"

namespace fmm {
cudaError_t launch_staged_f32(int mode, int vpl_mult, int stages, const PassArgs &a,
                              cudaStream_t st)
{
    return launch_staged_typed<float>(mode, vpl_mult, stages, a, st);
}
}  // namespace fmm
