// float32 instantiations of the row-pass kernels.
#include "fmm_rows.cuh"

namespace fmm {
cudaError_t launch_pass_f32(int mode, int vpl_mult, int ng, int u, bool vec, const PassArgs &a,
                            cudaStream_t st)
{
    return launch_pass_typed<float>(mode, vpl_mult, ng, u, vec, a, st);
}
}  // namespace fmm
