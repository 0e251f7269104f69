// Gather-rate probe: fetches dense rows through an index list and does
// nothing else, so its time is the ceiling for the gather part of a row pass
// that walks the same index list (the same rows, in the same order, from the
// same table, whether the table lives in L2 or in DRAM).  Not part of the
// paper's method; a measurement aid for the row passes.
//
// A team of ROW_BYTES / 16 lanes fetches one row with one 16-byte load per
// lane (ld.global.nc, as the row passes do); each team keeps U rows in
// flight; the loaded words are folded with xor into a value that is stored
// only if it equals a constant, which keeps every load alive at the cost of
// one predicated store per thread.
#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

template <int ROW_BYTES, int U>
__global__ void __launch_bounds__(256) gather_probe_kernel(const uint4 *table, int64_t rows,
                                                           const int32_t *idx, int64_t count,
                                                           uint32_t *sink)
{
    constexpr int G = ROW_BYTES / 16;
    const int lig = threadIdx.x & (G - 1);
    const int64_t team = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t teams = (int64_t)gridDim.x * blockDim.x / G;
    uint32_t acc = 0;
    for (int64_t base = team * U; base < count; base += teams * U) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t k = base + u;
            q[u] = make_uint4(0u, 0u, 0u, 0u);
            if (k < count) {
                // clamped into the table: a bad index cannot read outside it
                const int64_t j = min(max((int64_t)__ldg(idx + k), (int64_t)0), rows - 1);
                q[u] = __ldg(table + j * G + lig);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            acc ^= q[u].x ^ q[u].y ^ q[u].z ^ q[u].w;
    }
    if (acc == 0x9e3779b9u)
        sink[0] = acc;
}

template <int ROW_BYTES>
static cudaError_t launch_probe(const void *table, int64_t rows, const int32_t *idx,
                                int64_t count, uint32_t *sink, cudaStream_t st)
{
    constexpr int U = 4;
    constexpr int G = ROW_BYTES / 16;
    const int64_t teams_needed = (count + U - 1) / U;
    const int64_t blocks = std::min<int64_t>((teams_needed * G + 255) / 256,
                                             (int64_t)sm_count() * 8);
    gather_probe_kernel<ROW_BYTES, U><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
        static_cast<const uint4 *>(table), rows, idx, count, sink);
    return cudaGetLastError();
}

}  // namespace fmm

using namespace fmm;

extern "C" int fmm_probe_gather(const void *table, int64_t rows, int32_t row_bytes,
                                const int32_t *idx, int64_t count, uint32_t *sink,
                                fmm_stream stream)
{
    if (rows < 0 || count < 0) {
        set_error_msg("negative size");
        return FMM_EINVAL;
    }
    if (count == 0)
        return FMM_OK;
    if (rows == 0 || !table || !idx || !sink ||
        (reinterpret_cast<uintptr_t>(table) & 15u)) {
        set_error_msg("table (16-byte aligned, at least one row), idx and sink are required");
        return FMM_EINVAL;
    }
    cudaError_t e;
    cudaStream_t st = (cudaStream_t)stream;
    switch (row_bytes) {
    case 64: e = launch_probe<64>(table, rows, idx, count, sink, st); break;
    case 128: e = launch_probe<128>(table, rows, idx, count, sink, st); break;
    case 256: e = launch_probe<256>(table, rows, idx, count, sink, st); break;
    case 512: e = launch_probe<512>(table, rows, idx, count, sink, st); break;
    default:
        set_error_msg("row_bytes must be 64, 128, 256 or 512");
        return FMM_EUNSUPPORTED;
    }
    if (e != cudaSuccess) {
        set_error("fmm_probe_gather launch", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}
