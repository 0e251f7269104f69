// bfloat16 instantiations of the staged row-pass kernels.
#include "fmm_staged.cuh"

namespace fmm {
cudaError_t launch_staged_bf16(int mode, int vpl_mult, int stages, const PassArgs &a,
                              cudaStream_t st)
{
    return launch_staged_typed<bf16_t>(mode, vpl_mult, stages, a, st);
}
}  // namespace fmm
