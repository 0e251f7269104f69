// bfloat16-input instantiations of the pipelined forward-role row passes.
#include "fmm_pipe.cuh"

namespace fmm {
cudaError_t launch_pipe_bf16(int mode, int vpl_mult, int u, int ring, int mb, int refill,
                            const PassArgs &a, cudaStream_t st)
{
    return launch_pipe_typed<bf16_t>(mode, vpl_mult, u, ring, mb, refill, a, st);
}
}  // namespace fmm
