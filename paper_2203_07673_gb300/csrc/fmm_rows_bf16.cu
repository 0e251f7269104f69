// bfloat16-input instantiations of the row-pass kernels (float32 accumulation).
#include "fmm_rows.cuh"

namespace fmm {
cudaError_t launch_pass_bf16(int mode, int vpl_mult, int ng, int u, bool vec, const PassArgs &a,
                            cudaStream_t st)
{
    return launch_pass_typed<bf16_t>(mode, vpl_mult, ng, u, vec, a, st);
}
}  // namespace fmm
