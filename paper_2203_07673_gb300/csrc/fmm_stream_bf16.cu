// bfloat16-input instantiations of the streaming forward-role row passes.
#include "fmm_stream.cuh"

namespace fmm {
cudaError_t launch_stream_bf16(int mode, int vpl_mult, int ring, int mb, const PassArgs &a,
                               cudaStream_t st)
{
    return launch_stream_typed<bf16_t>(mode, vpl_mult, ring, mb, a, st);
}
}  // namespace fmm
