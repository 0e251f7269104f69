// fmm_fusedmm_noalloc: FusedMMA without a plan and without any allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the product: code running inside a memory pool or arena that owns all of
// the device memory, a runtime that forbids cudaMalloc (and the implicit
// synchronisation it can cause) on its hot path, or a host library that is
// handed only its inputs and outputs.  fmm_plan_create allocates (S^T, the
// schedule, the partial rows), so those callers cannot use a plan.  This
// entry point computes the same FusedMMA as fmm_fusedmm from the CSR
// directly.  Its only scratch memory -- the chunk list and partial rows of
// long rows -- lives in the file-scope device array below, of fixed size.
//
// Scratch:  g_noalloc_scratch, 34,603,264 bytes per device (every device that
// loads this library's module holds it until the process exits):
//   header   256 B       two counters, cleared at the start of every call
//   chunks   64 Ki x 16 B  (row, begin, end) of each chunk of a long row
//   split    64 Ki x 16 B  (row, first chunk, chunk count) of each long row
//   partials 8 Mi floats   one partial output row per chunk
// Rows longer than ch nonzeros are split into chunks of ch, where
// ch = max(512, ceil(2 nnz / cap)) and cap = min(64 Ki, 8 Mi / r): every long
// row has more than ch nonzeros, so its ceil(deg / ch) chunks number fewer
// than 2 deg / ch, and all chunks together fewer than 2 nnz / ch <= cap.
// The partial rows of a long row are summed in chunk order, so results are
// deterministic.  r may be at most 65536 (FMM_EOVERFLOW otherwise).
//
// Every call uses the same array: calls that overlap on the GPU (two streams,
// or two host threads without ordering) race on it and give wrong results.
// Order them on one stream.  Every call looks up the array's device address
// with cudaGetSymbolAddress on the current device (no allocation); the first
// call on a device may load the library's module there, so make that first
// call before any stream capture.
#include <cstdio>

#include "fmm_rows.cuh"

namespace fmm {
namespace noalloc {

constexpr int32_t MAX_CHUNKS = 1 << 16;
constexpr int32_t MAX_SPLIT = 1 << 16;
constexpr int64_t PARTIAL_FLOATS = int64_t(1) << 23;
constexpr int32_t MAX_R = 1 << 16;
constexpr int32_t MIN_CHUNK = 512;
constexpr size_t HEADER_BYTES = 256;
constexpr size_t CHUNKS_OFF = HEADER_BYTES;
constexpr size_t SPLIT_OFF = CHUNKS_OFF + sizeof(int4) * MAX_CHUNKS;
constexpr size_t PARTIALS_OFF = SPLIT_OFF + sizeof(int4) * MAX_SPLIT;
constexpr size_t SCRATCH_BYTES = PARTIALS_OFF + sizeof(float) * PARTIAL_FLOATS;

struct Header {
    int32_t n_chunks;
    int32_t n_split;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

struct Args {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const float *s;
    const void *A;
    const void *B;
    float *out;
    int32_t m, n, r, ch;
    int32_t cap;            // chunk slots usable at this r
    int64_t nnz;
    Header *hdr;
    int4 *chunks;
    int4 *split;
    float *partials;
};

// A chunk descriptor is used only if it lies inside this call's pattern
// (slots not written by this call hold an earlier call's descriptors).
__device__ __forceinline__ bool chunk_ok(const Args &a, const int4 c)
{
    return c.x >= 0 && c.x < a.m && c.y >= 0 && c.z >= c.y && (int64_t)c.z <= a.nnz;
}

// Row range of `row`, or an empty range if row_ptr is not consistent there
// (memory safety only: results for malformed patterns are unspecified).
__device__ __forceinline__ void row_range(const Args &a, int row, int &beg, int &end)
{
    beg = __ldg(a.row_ptr + row);
    end = __ldg(a.row_ptr + row + 1);
    if (beg < 0 || end < beg || (int64_t)end > a.nnz) {
        beg = 0;
        end = 0;
    }
}

__global__ void setup_kernel(const Args a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.m; i += stride) {
        int beg, end;
        row_range(a, (int)i, beg, end);
        if (end - beg <= a.ch)
            continue;
        const int nc = (end - beg + a.ch - 1) / a.ch;
        const int first = atomicAdd(&a.hdr->n_chunks, nc);
        const int slot = atomicAdd(&a.hdr->n_split, 1);
        if (slot >= MAX_SPLIT)
            continue;   // only a malformed pattern gets here; combine stops at MAX_SPLIT
        if ((int64_t)first + nc > a.cap) {
            a.split[slot] = make_int4((int)i, 0, 0, 0);   // malformed pattern: row left zero
            continue;
        }
        a.split[slot] = make_int4((int)i, first, nc, 0);
        for (int c = 0; c < nc; ++c) {
            const int b = beg + c * a.ch;
            a.chunks[first + c] = make_int4((int)i, b, (int)min((int64_t)end, (int64_t)b + a.ch), 0);
        }
    }
}

// The FusedMMA accumulation of nonzeros [beg, end) of `row` into acc (one
// group of G lanes; every lane of the warp must call it).
template <typename T, int R, int U>
__device__ __forceinline__ void fused_range(const Args &a, int row, int beg, int end, bool active,
                                            int lig, float (&acc)[Shape<T, R>::E])
{
    using S = Shape<T, R>;
    constexpr int G = S::G, E = S::E;
    const T *A = static_cast<const T *>(a.A);
    const T *B = static_cast<const T *>(a.B);
    float lrow[E];
#pragma unroll
    for (int e = 0; e < E; ++e) { lrow[e] = 0.f; acc[e] = 0.f; }
    if (active)
        load_row<T, R, true>(A + (size_t)row * R, lig, lrow);
    const int iters = active ? (end - beg + U - 1) / U : 0;
    const int witers = (int)__reduce_max_sync(0xffffffffu, (unsigned)iters);
    for (int it = 0; it < witers; ++it) {
        const int p0 = beg + it * U;
        int jj[U];
        float sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = p0 + u;
            jj[u] = -1;
            sv[u] = 0.f;
            if (active && p < end) {
                const int j = __ldg(a.col_idx + p);
                if (j >= 0 && j < a.n) {
                    jj[u] = j;
                    sv[u] = a.s ? __ldg(a.s + p) : 1.f;
                }
            }
        }
        float y[U][E];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                load_row<T, R, false>(B + (size_t)jj[u] * R, lig, y[u]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) y[u][e] = 0.f;
            }
        }
        float d[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float t = 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) t = fmaf(lrow[e], y[u][e], t);
            d[u] = t;
        }
        group_allreduce<G, U>(d);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0) continue;
            const float c = sv[u] * d[u];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = fmaf(c, y[u][e], acc[e]);
        }
    }
}

template <typename T, int R, int U>
__global__ void __launch_bounds__(256) rows_kernel(const Args a)
{
    constexpr int G = Shape<T, R>::G, E = Shape<T, R>::E;
    const int lig = threadIdx.x & (G - 1);
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    int row = 0, beg = 0, end = 0;
    bool active = gid < a.m;
    if (active) {
        row = (int)gid;
        row_range(a, row, beg, end);
        if (end - beg > a.ch)
            active = false;   // a long row: done by chunks_kernel
    }
    float acc[E];
    fused_range<T, R, U>(a, row, beg, end, active, lig, acc);
    if (active)
        store_row_f32<T, R>(a.out + (size_t)row * R, lig, acc);
}

template <typename T, int R, int U>
__global__ void __launch_bounds__(256) chunks_kernel(const Args a)
{
    constexpr int G = Shape<T, R>::G, E = Shape<T, R>::E;
    const int lig = threadIdx.x & (G - 1);
    const int n_chunks = min(a.hdr->n_chunks, a.cap);
    const long long groups = (long long)gridDim.x * blockDim.x / G;
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long rounds = (n_chunks + groups - 1) / groups;   // the same for every warp
    for (long long rd = 0; rd < rounds; ++rd) {
        const long long item = rd * groups + gid;
        bool active = item < n_chunks;
        int4 c = make_int4(0, 0, 0, 0);
        if (active) {
            c = a.chunks[item];
            if (!chunk_ok(a, c)) {
                active = false;
                c = make_int4(0, 0, 0, 0);
            }
        }
        float acc[E];
        fused_range<T, R, U>(a, c.x, c.y, c.z, active, lig, acc);
        if (active)
            store_row_f32<T, R>(a.partials + (size_t)item * R, lig, acc);
    }
}

// Any r, any alignment: one warp per row or chunk, the output row
// accumulated in place (lane k owns columns k, k + 32, ...).
template <typename T>
__device__ void generic_range(const Args &a, int row, int beg, int end, float *dst)
{
    const int lane = threadIdx.x & 31;
    const int r = a.r;
    const T *Ai = static_cast<const T *>(a.A) + (size_t)row * r;
    const T *B = static_cast<const T *>(a.B);
    for (int k = lane; k < r; k += 32)
        dst[k] = 0.f;
    for (int p = beg; p < end; ++p) {
        const int j = __ldg(a.col_idx + p);
        if (j < 0 || j >= a.n)
            continue;   // uniform across the warp
        const float sv = a.s ? __ldg(a.s + p) : 1.f;
        const T *Bj = B + (size_t)j * r;
        float d = 0.f;
        for (int k = lane; k < r; k += 32)
            d = fmaf(widen<T>(Ai[k]), widen<T>(Bj[k]), d);
        d = warp_allreduce(d);
        const float c = sv * d;
        for (int k = lane; k < r; k += 32)
            dst[k] = fmaf(c, widen<T>(Bj[k]), dst[k]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) rows_generic(const Args a)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= a.m)
        return;
    int beg, end;
    row_range(a, (int)w, beg, end);
    if (end - beg > a.ch)
        return;
    generic_range<T>(a, (int)w, beg, end, a.out + (size_t)w * a.r);
}

template <typename T>
__global__ void __launch_bounds__(256) chunks_generic(const Args a)
{
    const int n_chunks = min(a.hdr->n_chunks, a.cap);
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long item = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < n_chunks;
         item += warps) {
        const int4 c = a.chunks[item];
        if (!chunk_ok(a, c))
            continue;
        generic_range<T>(a, c.x, c.y, c.z, a.partials + (size_t)item * a.r);
    }
}

__global__ void combine_kernel(const Args a)
{
    const int n_split = min(a.hdr->n_split, MAX_SPLIT);
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_split;
         w += warps) {
        const int4 sp = a.split[w];
        if (sp.x < 0 || sp.x >= a.m || sp.y < 0 || sp.z < 0 || (int64_t)sp.y + sp.z > a.cap)
            continue;
        for (int k = lane; k < a.r; k += 32) {
            float acc = 0.f;
            for (int c = 0; c < sp.z; ++c)
                acc += a.partials[(size_t)(sp.y + c) * a.r + k];
            a.out[(size_t)sp.x * a.r + k] = acc;
        }
    }
}

template <typename T, int R>
void launch_vec(const Args &a, cudaStream_t st)
{
    constexpr int G = Shape<T, R>::G;
    constexpr int U = Shape<T, R>::E <= 4 ? 8 : 4;
    const long long blocks = ((long long)a.m * G + 255) / 256;
    if (blocks > 0)
        rows_kernel<T, R, U><<<(unsigned)blocks, 256, 0, st>>>(a);
    chunks_kernel<T, R, U><<<sm_count() * 8, 256, 0, st>>>(a);
}

template <typename T>
void launch_typed(const Args &a, bool vec, cudaStream_t st)
{
    if (vec) {
        switch (a.r) {
        case 32: launch_vec<T, 32>(a, st); return;
        case 64: launch_vec<T, 64>(a, st); return;
        case 128: launch_vec<T, 128>(a, st); return;
        case 256: launch_vec<T, 256>(a, st); return;
        default: break;
        }
    }
    const long long blocks = ((long long)a.m + 7) / 8;
    if (blocks > 0)
        rows_generic<T><<<(unsigned)blocks, 256, 0, st>>>(a);
    chunks_generic<T><<<sm_count() * 8, 256, 0, st>>>(a);
}

// The array's device address, looked up on every call with the current
// device (cudaGetSymbolAddress allocates nothing).  Nothing is cached, so a
// module reloaded at another address (after cudaDeviceReset) is followed.
int scratch_base(unsigned char **base)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(no-alloc scratch)", e);
        return FMM_ECUDA;
    }
    *base = static_cast<unsigned char *>(p);
    return FMM_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace noalloc
}  // namespace fmm

extern "C" int fmm_fusedmm_noalloc(const fmm_csr *S, int32_t r, int32_t dtype, const float *vals,
                                   const void *A, const void *B, float *out_m, fmm_stream stream)
{
    using namespace fmm;
    using namespace fmm::noalloc;
    int rc = check_csr_args(S);
    if (rc)
        return rc;
    if (r < 1 || (dtype != FMM_F32 && dtype != FMM_BF16)) {
        set_error_msg("r must be >= 1 and dtype FMM_F32 or FMM_BF16");
        return FMM_EUNSUPPORTED;
    }
    if (r > MAX_R) {
        set_error_msg("r exceeds the no-alloc maximum of 65536");
        return FMM_EOVERFLOW;
    }
    if ((S->m > 0 && (!A || !out_m)) || (S->n > 0 && !B)) {
        set_error_msg("A, B or out_m is NULL");
        return FMM_EINVAL;
    }
    if (S->m == 0)
        return FMM_OK;
    unsigned char *base = nullptr;
    rc = scratch_base(&base);
    if (rc)
        return rc;
    const int64_t cap = std::min<int64_t>(MAX_CHUNKS, PARTIAL_FLOATS / r);
    const int64_t ch = std::max<int64_t>(MIN_CHUNK, (2 * S->nnz + cap - 1) / cap);
    Args a;
    a.row_ptr = S->row_ptr;
    a.col_idx = S->col_idx;
    a.s = vals;
    a.A = A;
    a.B = B;
    a.out = out_m;
    a.m = S->m;
    a.n = S->n;
    a.r = r;
    a.ch = (int32_t)std::min<int64_t>(ch, INT32_MAX);
    a.cap = (int32_t)cap;
    a.nnz = S->nnz;
    a.hdr = reinterpret_cast<Header *>(base);
    a.chunks = reinterpret_cast<int4 *>(base + CHUNKS_OFF);
    a.split = reinterpret_cast<int4 *>(base + SPLIT_OFF);
    a.partials = reinterpret_cast<float *>(base + PARTIALS_OFF);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(base, 0, HEADER_BYTES, st);
    if (e == cudaSuccess) {
        const long long blocks = std::min<long long>(((long long)S->m + 255) / 256, (long long)sm_count() * 16);
        setup_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
        const bool vec = fast_r(r) && aligned16(A) && aligned16(B) && aligned16(out_m);
        if (dtype == FMM_BF16)
            launch_typed<bf16_t>(a, vec, st);
        else
            launch_typed<float>(a, vec, st);
        combine_kernel<<<sm_count() * 4, 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fmm_fusedmm_noalloc launch", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}
