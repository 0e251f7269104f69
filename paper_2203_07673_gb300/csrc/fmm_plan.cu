// Plan construction: validation of the pattern, the transposed pattern with
// its permutation (stable LSD radix sort by column), and the schedule of each
// side (rows ordered by length, long rows split into fixed-size chunks).
//
// The transposed copy of S is how the paper obtains FusedMMB and SpMMB from
// the FusedMMA machinery: interchange A and B and use S^T, "storing two
// copies of the sparse matrix, one with the coordinates transposed"
// (Sec. IV-B, last paragraph).  Preprocessing the pattern once and reusing it
// over repeated calls with the same nonzero structure follows Sec. I and
// Sec. III-A.  All of it runs on the device; the host only sizes buffers and
// lays out the (few) chunks of split rows.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

// ---------------------------------------------------------------- validation

__global__ void validate_kernel(const int32_t *row_ptr, const int32_t *col_idx, int32_t m,
                                int32_t n, int64_t nnz, unsigned long long *bad_rp,
                                unsigned long long *bad_ci)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= (int64_t)m; i += stride) {
        const int64_t v = row_ptr[i];
        bool bad = v < 0 || v > nnz;
        if (i == 0 && v != 0) bad = true;
        if (i == m && v != nnz) bad = true;
        if (i > 0 && v < (int64_t)row_ptr[i - 1]) bad = true;
        if (bad)
            atomicMin(bad_rp, (unsigned long long)i);
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        const int32_t c = col_idx[p];
        if (c < 0 || c >= n)
            atomicMin(bad_ci, (unsigned long long)p);
    }
}

// ------------------------------------------------------------------ scan

// Exclusive prefix sum of n uint32 values (in may equal out), one block of
// 1024 threads walking the array in tiles of 4096 with a running carry.
__global__ void __launch_bounds__(1024) scan_exclusive_kernel(const uint32_t *in, uint32_t *out,
                                                              int64_t n)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0)
        carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 4096) {
        uint32_t x[4], sum = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t idx = base + tid * 4 + t;
            x[t] = idx < n ? in[idx] : 0u;
            sum += x[t];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31)
            warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint32_t t = warp_tot[lane], ti = t;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, ti, off);
                if (lane >= off) ti += y;
            }
            warp_tot[lane] = ti - t;   // exclusive over warps
        }
        __syncthreads();
        uint32_t run = carry_s + warp_tot[w] + (incl - sum);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t idx = base + tid * 4 + t;
            if (idx < n)
                out[idx] = run;
            run += x[t];
        }
        __syncthreads();
        if (tid == 1023)
            carry_s = run;
        __syncthreads();
    }
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) pairs, 8-bit digits, tiles of 4096
// items (256 threads x 16).  Each warp owns 512 consecutive items of a tile
// and ranks them in order with __match_any_sync, so equal digits keep their
// input order: the sort is stable and fully deterministic.

constexpr int RS_TILE = 4096;

__global__ void __launch_bounds__(256) rs_hist_kernel(const uint32_t *keys, int64_t n, int shift,
                                                      uint32_t *ghist, int ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int t = 0; t < 16; ++t) {
        const int64_t idx = base + t * 256 + threadIdx.x;
        if (idx < n)
            atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    ghist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(256) rs_scatter_kernel(const uint32_t *kin, const int32_t *vin,
                                                         uint32_t *kout, int32_t *vout, int64_t n,
                                                         int shift, const uint32_t *goff,
                                                         int ntiles)
{
    __shared__ uint32_t wc[8][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + w * 512;
    uint32_t key[16];
    int32_t val[16];
    int dig[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const int64_t idx = base + t * 32 + lane;
        if (idx < n) {
            key[t] = kin[idx];
            val[t] = vin[idx];
            dig[t] = (int)((key[t] >> shift) & 255u);
        } else {
            key[t] = 0; val[t] = 0; dig[t] = 256;
        }
    }
    for (int i = tid; i < 8 * 256; i += 256)
        (&wc[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[t]);
        const int leader = 31 - __clz(peers);
        if (dig[t] < 256 && lane == leader)
            wc[w][dig[t]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = goff[(size_t)tid * ntiles + blockIdx.x];
        for (int w2 = 0; w2 < 8; ++w2) {
            const uint32_t c = wc[w2][tid];
            wc[w2][tid] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[t]);
        const int leader = 31 - __clz(peers);
        if (dig[t] < 256) {
            const uint32_t pos = wc[w][dig[t]] + __popc(peers & lt);
            kout[pos] = key[t];
            vout[pos] = val[t];
        }
        __syncwarp();
        if (dig[t] < 256 && lane == leader)
            wc[w][dig[t]] += __popc(peers);
        __syncwarp();
    }
}

static int blocks_for(int64_t n, int threads, int cap = 1 << 20)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

// Sorts by the low `bits` bits of the keys; on return *in_b says whether the
// result sits in (kb, vb) rather than (ka, va).
static cudaError_t radix_sort(uint32_t *ka, int32_t *va, uint32_t *kb, int32_t *vb, int64_t n,
                              int bits, uint32_t *ghist, cudaStream_t st, bool *in_b)
{
    *in_b = false;
    if (n <= 1)
        return cudaSuccess;
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    uint32_t *ks = ka, *kd = kb;
    int32_t *vs = va, *vd = vb;
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<ntiles, 256, 0, st>>>(ks, n, shift, ghist, ntiles);
        scan_exclusive_kernel<<<1, 1024, 0, st>>>(ghist, ghist, (int64_t)ntiles * 256);
        rs_scatter_kernel<<<ntiles, 256, 0, st>>>(ks, vs, kd, vd, n, shift, ghist, ntiles);
        std::swap(ks, kd);
        std::swap(vs, vd);
        *in_b = !*in_b;
    }
    return cudaGetLastError();
}

// --------------------------------------------------------- side schedule

// Sort key of every row (length_key) and the counts of split rows and the
// longest row.
__global__ void row_keys_kernel(const int32_t *row_ptr, int32_t rows, int32_t split_nnz,
                                uint32_t *keys, int32_t *vals, int32_t *counters)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += stride) {
        const int32_t deg = row_ptr[i + 1] - row_ptr[i];
        const uint32_t key = length_key(deg, split_nnz);
        if (key == 0)
            atomicAdd(&counters[0], 1);
        atomicMax(&counters[1], deg);
        keys[i] = key;
        vals[i] = (int32_t)i;
    }
}

__global__ void split_ranges_kernel(const int32_t *order, int32_t n_split, const int32_t *row_ptr,
                                    int2 *ranges)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_split; i += stride) {
        const int32_t row = order[i];
        ranges[i] = make_int2(row_ptr[row], row_ptr[row + 1]);
    }
}

// ----------------------------------------------------------- transpose

__global__ void count_cols_kernel(const int32_t *col_idx, int64_t nnz, uint32_t *cnt)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
        atomicAdd(&cnt[col_idx[p]], 1u);
}

__global__ void init_pairs_kernel(const int32_t *col_idx, int64_t nnz, uint32_t *keys,
                                  int32_t *vals)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        keys[p] = (uint32_t)col_idx[p];
        vals[p] = (int32_t)p;
    }
}

// col_idx_t[q] = the row of S holding nonzero perm[q] (binary search in row_ptr).
__global__ void rows_of_kernel(const int32_t *row_ptr, int32_t m, const int32_t *perm,
                               int32_t *col_idx_t, int64_t nnz)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
        const int32_t p = perm[q];
        int32_t lo = 0, hi = m - 1;
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo + 1) / 2;
            if (row_ptr[mid] <= p) lo = mid; else hi = mid - 1;
        }
        col_idx_t[q] = lo;
    }
}

// Windowed value permutation, plan time.  Window w holds the S^T slots
// [w P, (w + 1) P).  key[perm[q]] = q / P (the window of each S slot's
// destination), val[p] = p; a stable sort by key lists, per window, its
// source slots in S order, so sorted position i of slot p is pos1[p]; then
// pos2[q] = pos1[perm[q]] is where the value of S^T slot q waits in pass 2.
__global__ void window_keys_kernel(const int32_t *perm, int64_t nnz, int64_t P, uint32_t *keys,
                                   int32_t *vals)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
        keys[perm[q]] = (uint32_t)(q / P);
        vals[q] = (int32_t)q;
    }
}

__global__ void window_pos1_kernel(const int32_t *sorted_slots, int64_t nnz, int32_t *pos1)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride)
        pos1[sorted_slots[i]] = (int32_t)i;
}

__global__ void window_pos2_kernel(const int32_t *perm, const int32_t *pos1, int64_t nnz,
                                   int32_t *pos2)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride)
        pos2[q] = pos1[perm[q]];
}

}  // namespace fmm

// ====================================================================== API

using namespace fmm;

namespace {

thread_local char g_last_error[256] = "";

struct Temps {
    uint32_t *ka = nullptr, *kb = nullptr, *ghist = nullptr;
    int32_t *va = nullptr, *vb = nullptr, *counters = nullptr;
    ~Temps()
    {
        cudaFree(ka); cudaFree(kb); cudaFree(ghist);
        cudaFree(va); cudaFree(vb); cudaFree(counters);
    }
};

}  // namespace

namespace fmm {

void set_error(const char *what, cudaError_t e)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what,
             e == cudaSuccess ? "ok" : cudaGetErrorString(e));
}

void set_error_msg(const char *what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s", what);
}

const char *last_error() { return g_last_error; }

template <typename P>
static cudaError_t dmalloc(P **p, size_t count, fmm_plan *plan)
{
    size_t bytes = count * sizeof(P);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess && plan) plan->workspace_bytes += (int64_t)bytes;
    return e;
}

#define FMM_TRY(expr, what)                                          \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) {                                     \
            set_error(what, _e);                                     \
            return _e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA; \
        }                                                            \
    } while (0)

// Runs of the streaming pass (host, once per side): consecutive light rows
// (at most split_nnz nonzeros) taken greedily in index order while the run
// stays within kRunNnz nonzeros and kRunRows rows; a split row ends a run
// and belongs to none (its chunks are work items of their own).  Runs are
// ordered by nonzero count, longest first (stable), so the teams of one warp
// walk streams of similar length.
static int build_runs(Side &side, const int32_t *row_ptr, int32_t rows, int32_t split_nnz,
                      cudaStream_t st, fmm_plan *plan)
{
    std::vector<int32_t> rp((size_t)rows + 1);
    FMM_TRY(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int32_t) * ((size_t)rows + 1),
                            cudaMemcpyDeviceToHost, st), "read row pointers");
    FMM_TRY(cudaStreamSynchronize(st), "plan sync");
    std::vector<int2> runs;
    std::vector<int32_t> nnz;
    int32_t start = -1, count = 0, rows_in = 0;
    auto close = [&](int32_t end) {
        if (start >= 0) {
            runs.push_back(make_int2(start, end));
            nnz.push_back(count);
        }
        start = -1; count = 0; rows_in = 0;
    };
    for (int32_t i = 0; i < rows; ++i) {
        const int32_t d = rp[i + 1] - rp[i];
        if (d > split_nnz) {
            close(i);
            continue;
        }
        if (start >= 0 && (count + d > kRunNnz || rows_in == kRunRows))
            close(i);
        if (start < 0)
            start = i;
        count += d;
        ++rows_in;
    }
    close(rows);
    std::vector<int32_t> idx(runs.size());
    for (size_t k = 0; k < idx.size(); ++k)
        idx[k] = (int32_t)k;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return nnz[x] > nnz[y]; });
    std::vector<int2> sorted(runs.size());
    for (size_t k = 0; k < idx.size(); ++k)
        sorted[k] = runs[idx[k]];
    side.n_runs = (int32_t)sorted.size();
    if (side.n_runs == 0)
        return FMM_OK;
    FMM_TRY(dmalloc(&side.runs, sorted.size(), plan), "allocate runs");
    FMM_TRY(cudaMemcpyAsync(side.runs, sorted.data(), sizeof(int2) * sorted.size(),
                            cudaMemcpyHostToDevice, st), "upload runs");
    FMM_TRY(cudaStreamSynchronize(st), "plan sync");
    return FMM_OK;
}

static int build_side(Side &side, const int32_t *row_ptr, int32_t rows, int32_t split_nnz,
                      int32_t r, Temps &tmp, cudaStream_t st, fmm_plan *plan)
{
    side.rows = rows;
    side.row_ptr = row_ptr;
    if (rows == 0)
        return FMM_OK;
    FMM_TRY(dmalloc(&side.order, (size_t)rows, plan), "allocate row order");
    FMM_TRY(cudaMemsetAsync(tmp.counters, 0, 2 * sizeof(int32_t), st), "memset");
    row_keys_kernel<<<blocks_for(rows, 256), 256, 0, st>>>(row_ptr, rows, split_nnz, tmp.ka,
                                                           tmp.va, tmp.counters);
    FMM_TRY(cudaGetLastError(), "row keys");
    bool in_b = false;
    FMM_TRY(radix_sort(tmp.ka, tmp.va, tmp.kb, tmp.vb, rows, 8, tmp.ghist, st, &in_b),
            "row order sort");
    FMM_TRY(cudaMemcpyAsync(side.order, in_b ? tmp.vb : tmp.va, (size_t)rows * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, st), "copy row order");
    // start of every length key in `order`: the scanned digit offsets of the
    // sort's first tile (entry key * ntiles of the histogram)
    side.bucket_start.assign(257, 0);
    if (rows > 1) {
        const int64_t ntiles = (rows + RS_TILE - 1) / RS_TILE;
        uint32_t starts[256];
        FMM_TRY(cudaMemcpy2DAsync(starts, sizeof(uint32_t), tmp.ghist, ntiles * sizeof(uint32_t),
                                  sizeof(uint32_t), 256, cudaMemcpyDeviceToHost, st),
                "read bucket starts");
        FMM_TRY(cudaStreamSynchronize(st), "plan sync");
        for (int k = 0; k < 256; ++k)
            side.bucket_start[k] = (int32_t)starts[k];
    } else {
        // a single row: its key decides its bucket (computed below from max_nnz)
        side.bucket_start.assign(257, rows);
    }
    side.bucket_start[256] = rows;
    int32_t counters[2];
    FMM_TRY(cudaMemcpyAsync(counters, tmp.counters, sizeof(counters), cudaMemcpyDeviceToHost, st),
            "read counters");
    FMM_TRY(cudaStreamSynchronize(st), "plan sync");
    side.n_split = counters[0];
    side.max_nnz = counters[1];
    side.n_light = rows - side.n_split;
    if (rows == 1) {
        const int key = (int)length_key(side.max_nnz, split_nnz);
        for (int k = 0; k <= key; ++k)
            side.bucket_start[k] = 0;
    }
    {
        const int rc = build_runs(side, row_ptr, rows, split_nnz, st, plan);
        if (rc != FMM_OK)
            return rc;
    }
    if (side.n_split == 0)
        return FMM_OK;
    int2 *d_ranges = nullptr;
    FMM_TRY(cudaMalloc(&d_ranges, sizeof(int2) * side.n_split), "allocate ranges");
    split_ranges_kernel<<<blocks_for(side.n_split, 256), 256, 0, st>>>(side.order, side.n_split,
                                                                       row_ptr, d_ranges);
    std::vector<int2> ranges(side.n_split);
    std::vector<int32_t> rows_h(side.n_split);
    cudaError_t e = cudaMemcpyAsync(ranges.data(), d_ranges, sizeof(int2) * side.n_split,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rows_h.data(), side.order, sizeof(int32_t) * side.n_split,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(d_ranges);
    FMM_TRY(e, "read split rows");
    std::vector<int4> chunks, split;
    for (int32_t s = 0; s < side.n_split; ++s) {
        const int32_t beg = ranges[s].x, end = ranges[s].y;
        const int32_t first = (int32_t)chunks.size();
        for (int64_t c = beg; c < end; c += split_nnz)
            chunks.push_back(make_int4(rows_h[s], (int32_t)c,
                                       (int32_t)std::min<int64_t>(end, c + split_nnz), 0));
        split.push_back(make_int4(rows_h[s], first, (int32_t)chunks.size() - first, 0));
    }
    side.n_chunks = (int32_t)chunks.size();
    FMM_TRY(dmalloc(&side.chunks, chunks.size(), plan), "allocate chunks");
    FMM_TRY(dmalloc(&side.split, split.size(), plan), "allocate split table");
    // three partial rows per chunk: the FusedMM passes use the first
    // n_chunks x r floats; the attention pass also keeps its running softmax
    // maximum and sum per element there
    FMM_TRY(dmalloc(&side.partials, (size_t)side.n_chunks * r * 3, plan), "allocate partials");
    FMM_TRY(cudaMemcpyAsync(side.chunks, chunks.data(), sizeof(int4) * chunks.size(),
                            cudaMemcpyHostToDevice, st), "upload chunks");
    FMM_TRY(cudaMemcpyAsync(side.split, split.data(), sizeof(int4) * split.size(),
                            cudaMemcpyHostToDevice, st), "upload split table");
    FMM_TRY(cudaStreamSynchronize(st), "plan sync");
    return FMM_OK;
}

static void free_side(Side &s)
{
    cudaFree(s.order); cudaFree(s.chunks); cudaFree(s.split); cudaFree(s.partials);
    cudaFree(s.runs);
    s = Side();
}

int check_csr_args(const fmm_csr *S)
{
    if (!S) { set_error_msg("S is NULL"); return FMM_EINVAL; }
    if (S->m < 0 || S->n < 0 || S->nnz < 0) { set_error_msg("negative size"); return FMM_EINVAL; }
    if (S->nnz >= (int64_t(1) << 31)) { set_error_msg("nnz >= 2^31"); return FMM_EOVERFLOW; }
    if (!S->row_ptr) { set_error_msg("row_ptr is NULL"); return FMM_EINVAL; }
    if (S->nnz > 0 && !S->col_idx) { set_error_msg("col_idx is NULL"); return FMM_EINVAL; }
    return FMM_OK;
}

int validate_csr(const fmm_csr *S, cudaStream_t st, int64_t *first_bad)
{
    if (first_bad) *first_bad = -1;
    unsigned long long *d_bad = nullptr;
    FMM_TRY(cudaMalloc(&d_bad, 2 * sizeof(unsigned long long)), "allocate validation flags");
    const unsigned long long init[2] = {~0ull, ~0ull};
    unsigned long long bad[2] = {~0ull, ~0ull};
    cudaError_t e = cudaMemcpyAsync(d_bad, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int64_t work = std::max<int64_t>((int64_t)S->m + 1, S->nnz);
        validate_kernel<<<blocks_for(work, 256, sm_count() * 16), 256, 0, st>>>(
            S->row_ptr, S->col_idx, S->m, S->n, S->nnz, d_bad, d_bad + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(d_bad);
    FMM_TRY(e, "validate CSR");
    if (bad[0] != ~0ull) {
        if (first_bad) *first_bad = -(int64_t)bad[0] - 2;
        snprintf(g_last_error, sizeof(g_last_error), "malformed CSR: row_ptr[%llu]", bad[0]);
        return FMM_EINVAL;
    }
    if (bad[1] != ~0ull) {
        if (first_bad) *first_bad = (int64_t)bad[1];
        snprintf(g_last_error, sizeof(g_last_error), "malformed CSR: col_idx[%llu] out of range",
                 bad[1]);
        return FMM_EINVAL;
    }
    return FMM_OK;
}

void destroy_plan(fmm_plan *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    free_side(p->rows);
    free_side(p->cols);
    cudaFree(p->row_ptr_t);
    cudaFree(p->col_idx_t);
    cudaFree(p->perm_t);
    cudaFree(p->vals_t);
    cudaFree(p->vals_static);
    cudaFree(p->win_pos1);
    cudaFree(p->win_pos2);
    cudaFree(p->win_tmp);
    cudaFree(p->err);
    delete p;
}

int create_plan(const fmm_csr *S, int32_t r, int32_t dtype, const fmm_plan_options *opt,
                cudaStream_t st, fmm_plan **out)
{
    fmm_plan *p = new fmm_plan();
    p->m = S->m; p->n = S->n; p->nnz = S->nnz; p->r = r; p->dtype = dtype;
    p->flags = opt ? opt->flags : 0u;
    if (opt) p->variant = opt->variant;
    const KernelVariant row_variant =
        p->variant ? decode_variant(p->variant)
                   : default_variant(r, dtype, S->m ? (double)S->nnz / S->m : 0.0);
    p->split_nnz = default_split_nnz(S->nnz, r, dtype, row_variant);
    if (opt && opt->split_nnz > 0) p->split_nnz = opt->split_nnz;
    cudaGetDevice(&p->device);
    Temps tmp;
    const int64_t N = std::max<int64_t>({(int64_t)S->m, (int64_t)S->n, S->nnz, 1});
    const int64_t ntiles = (N + RS_TILE - 1) / RS_TILE;
    int rc = FMM_OK;
    auto fail = [&](int code) { destroy_plan(p); *out = nullptr; return code; };
#define PLAN_TRY(expr, what)                                                    \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) {                                                \
            set_error(what, _e);                                                \
            return fail(_e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA); \
        }                                                                       \
    } while (0)
    PLAN_TRY(dmalloc(&tmp.ka, N, nullptr), "allocate sort keys");
    PLAN_TRY(dmalloc(&tmp.kb, N, nullptr), "allocate sort keys");
    PLAN_TRY(dmalloc(&tmp.va, N, nullptr), "allocate sort values");
    PLAN_TRY(dmalloc(&tmp.vb, N, nullptr), "allocate sort values");
    PLAN_TRY(dmalloc(&tmp.ghist, (size_t)ntiles * 256, nullptr), "allocate histogram");
    PLAN_TRY(dmalloc(&tmp.counters, 2, nullptr), "allocate counters");
    PLAN_TRY(dmalloc(&p->err, 1, p), "allocate error word");
    PLAN_TRY(cudaMemsetAsync(p->err, 0, sizeof(int32_t), st), "clear error word");

    rc = build_side(p->rows, S->row_ptr, S->m, p->split_nnz, r, tmp, st, p);
    if (rc) return fail(rc);
    p->rows.col_idx = S->col_idx;
    p->rows.perm = nullptr;
    p->rows.variant = row_variant;

    if (!(p->flags & FMM_PLAN_NO_TRANSPOSE)) {
        p->has_t = true;
        PLAN_TRY(dmalloc(&p->row_ptr_t, (size_t)S->n + 1, p), "allocate S^T row_ptr");
        PLAN_TRY(dmalloc(&p->col_idx_t, (size_t)S->nnz, p), "allocate S^T col_idx");
        PLAN_TRY(dmalloc(&p->perm_t, (size_t)S->nnz, p), "allocate S^T perm");
        uint32_t *cnt = reinterpret_cast<uint32_t *>(p->row_ptr_t);
        PLAN_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * ((size_t)S->n + 1), st), "memset");
        if (S->nnz > 0) {
            count_cols_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(S->col_idx,
                                                                                 S->nnz, cnt);
            init_pairs_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(
                S->col_idx, S->nnz, tmp.ka, tmp.va);
            PLAN_TRY(cudaGetLastError(), "transpose setup");
        }
        scan_exclusive_kernel<<<1, 1024, 0, st>>>(cnt, cnt, (int64_t)S->n + 1);
        PLAN_TRY(cudaGetLastError(), "transpose scan");
        int bits = 0;
        while (bits < 31 && (int64_t(1) << bits) < (int64_t)S->n) ++bits;
        bool in_b = false;
        if (S->nnz > 0) {
            PLAN_TRY(radix_sort(tmp.ka, tmp.va, tmp.kb, tmp.vb, S->nnz, bits, tmp.ghist, st, &in_b),
                     "transpose sort");
            PLAN_TRY(cudaMemcpyAsync(p->perm_t, in_b ? tmp.vb : tmp.va,
                                     sizeof(int32_t) * (size_t)S->nnz, cudaMemcpyDeviceToDevice, st),
                     "copy perm");
            rows_of_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(
                S->row_ptr, S->m, p->perm_t, p->col_idx_t, S->nnz);
            PLAN_TRY(cudaGetLastError(), "transpose rows");
        }
        PLAN_TRY(dmalloc(&p->vals_t, (size_t)S->nnz, p), "allocate S^T values");
        if (S->nnz > 2 * kPermuteWindow) {
            // the windowed value permutation (launch_values_t)
            const int64_t P = kPermuteWindow;
            const int64_t W = (S->nnz + P - 1) / P;
            int wbits = 0;
            while ((int64_t(1) << wbits) < W) ++wbits;
            PLAN_TRY(dmalloc(&p->win_pos1, (size_t)S->nnz, p), "allocate window positions");
            PLAN_TRY(dmalloc(&p->win_pos2, (size_t)S->nnz, p), "allocate window positions");
            PLAN_TRY(dmalloc(&p->win_tmp, (size_t)S->nnz, p), "allocate window values");
            window_keys_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(
                p->perm_t, S->nnz, P, tmp.ka, tmp.va);
            PLAN_TRY(cudaGetLastError(), "window keys");
            bool wb = false;
            PLAN_TRY(radix_sort(tmp.ka, tmp.va, tmp.kb, tmp.vb, S->nnz, wbits, tmp.ghist, st, &wb),
                     "window sort");
            window_pos1_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(
                wb ? tmp.vb : tmp.va, S->nnz, p->win_pos1);
            window_pos2_kernel<<<blocks_for(S->nnz, 256, sm_count() * 32), 256, 0, st>>>(
                p->perm_t, p->win_pos1, S->nnz, p->win_pos2);
            PLAN_TRY(cudaGetLastError(), "window positions");
        }
        rc = build_side(p->cols, p->row_ptr_t, S->n, p->split_nnz, r, tmp, st, p);
        if (rc) return fail(rc);
        p->cols.col_idx = p->col_idx_t;
        p->cols.perm = p->perm_t;
        p->cols.variant = p->variant ? decode_variant(p->variant)
                                     : default_variant(r, dtype, S->n ? (double)S->nnz / S->n : 0.0);
    } else {
        p->cols.max_nnz = -1;
    }
    PLAN_TRY(cudaStreamSynchronize(st), "plan sync");
#undef PLAN_TRY
    *out = p;
    return FMM_OK;
}

// Measured on GB300 over ER (32 per row), R-MAT and Zipf-row patterns at
// r = 64 and 128, FP32 and BF16, forward and both backward passes: one group
// per output row, 8 elements (32 bytes) per lane and 2 nonzeros per batch is
// the best or within a few percent of it (the lighter register footprint
// keeps more rows in flight than deeper batches do).
KernelVariant team_default_variant(int32_t r, int32_t dtype)
{
    KernelVariant v;
    v.ng = 1;
    v.u = 2;
    const int vecs = r * (dtype == FMM_BF16 ? 2 : 4) / 16;
    // float32 rows of at most 32 vectors hold 4 elements per vector: two
    // vectors per lane make 8 elements
    v.vpl_mult = (dtype == FMM_F32 && vecs <= 32) ? 2 : 1;
    return v;
}

KernelVariant default_variant(int32_t r, int32_t dtype, double avg_nnz)
{
    (void)avg_nnz;
    KernelVariant v = team_default_variant(r, dtype);
    // bfloat16 rows of r = 64 and 128: the register-ring pass with 16
    // elements per lane, one nonzero per batch and the slot refilled as soon
    // as it is read (code 32212).  Measured on GB300 (FusedMMA / FusedMMB
    // pass, ms): Zipf rows 2^21 x 2^19 1.71 / 1.54 -> 1.36 / 1.06, R-MAT 2^22
    // 1.65 -> 1.41, Erdos-Renyi 2^20 at r = 128 1.55 / 1.74 -> 1.41 / 1.53.
    // Of the backward roles, the pass over S runs the same ring pass, the pass
    // over S^T the team kernel's default layout.
    if (dtype == FMM_BF16 && (r == 64 || r == 128)) {
        v.vpl_mult = 2;
        v.u = 1;
        v.ring = 2;
        v.mb = 2;
        v.refill = 1;
    }
    // float32 rows of r = 128 (512 bytes): the staged pass with a ring of 4
    // gathered rows per team, 3-4 % faster on Erdos-Renyi rows at the DRAM
    // roofline (it needs no register spill); where gathers mostly hit L2 the
    // extra trip through shared memory costs more than the deeper ring
    // gains, and the team kernel stays
    if (dtype == FMM_F32 && r == 128)
        v.stages = 4;
    return v;
}

// Split size of long rows.  Chunks are scheduled first, and one team works
// through a chunk U*NG nonzeros per dependent step, while all concurrent
// teams share the rest of the pass; a chunk must end well before the pass
// does, so it holds at most nnz / (4 x concurrent teams) nonzeros.  Teams
// at once: SMs x resident warps x teams per warp (32 / lanes per team of
// the variant; rows of the generic kernel take a warp); resident warps are
// 8 per requested block for the register-ring and bulk-staged passes, else
// 32.  Within [256, 8192].  (The register-ring pass on the Zipf-row pattern
// with bfloat16 rows of r = 64: chunks of 514 nonzeros took 1.51 ms, of
// 1028 1.37 ms.)
// (On R-MAT 2^22 with BF16 rows of r = 64 this gives about 840; chunks of
// 3982 made that forward pass 15 % slower than chunks of 1024.)
int32_t default_split_nnz(int64_t nnz, int32_t r, int32_t dtype, const KernelVariant &v)
{
    const int e = dtype == FMM_BF16 ? 2 : 4;
    int lanes = 32;
    if (fast_r(r)) {
        const int vecs = r * e / 16;
        const int vpl = (vecs > 32 ? vecs / 32 : 1) * v.vpl_mult;
        lanes = std::min(32, std::max(1, vecs / std::max(1, vpl)) * std::max(1, v.ng));
    }
    const int warps = (v.ring > 0 || v.depth > 0 || v.stream) && v.mb > 0 ? 8 * v.mb : 32;
    const int64_t teams = (int64_t)sm_count() * warps * (32 / lanes);
    return (int32_t)std::min<int64_t>(8192, std::max<int64_t>(256, nnz / (4 * teams)));
}

// dst[q] = src[perm[q]].  Each block covers 1024 consecutive q, each thread
// four of them 256 apart: the perm loads and the stores of a warp stay
// coalesced, and every thread has four independent gathers in flight.
// (One 16-byte perm load per thread for four adjacent q measured slower on
// patterns whose S^T visits S in long scattered runs.)
constexpr int kPermuteBlock = 256;
constexpr int kPermutePerThread = 4;

__global__ void __launch_bounds__(kPermuteBlock) permute_kernel(const float *src,
                                                               const int32_t *perm, float *dst,
                                                               int64_t nnz)
{
    const int64_t base =
        (int64_t)blockIdx.x * (kPermuteBlock * kPermutePerThread) + threadIdx.x;
    int32_t p[kPermutePerThread];
    float v[kPermutePerThread];
#pragma unroll
    for (int j = 0; j < kPermutePerThread; ++j) {
        const int64_t q = base + (int64_t)kPermuteBlock * j;
        p[j] = q < nnz ? __ldcs(perm + q) : 0;
    }
#pragma unroll
    for (int j = 0; j < kPermutePerThread; ++j) {
        const int64_t q = base + (int64_t)kPermuteBlock * j;
        v[j] = q < nnz ? __ldg(src + p[j]) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kPermutePerThread; ++j) {
        const int64_t q = base + (int64_t)kPermuteBlock * j;
        if (q < nnz)
            dst[q] = v[j];
    }
}

cudaError_t launch_permute(const float *src, const int32_t *perm, float *dst, int64_t nnz,
                           cudaStream_t st)
{
    if (nnz == 0 || !src)
        return cudaSuccess;
    const int64_t per_block = kPermuteBlock * kPermutePerThread;
    const int64_t blocks = (nnz + per_block - 1) / per_block;   // nnz < 2^31: < 2^21 blocks
    permute_kernel<<<(unsigned)blocks, kPermuteBlock, 0, st>>>(src, perm, dst, nnz);
    return cudaGetLastError();
}

// dst[pos[p]] = src[p]: the first pass of the windowed permutation.  Reads
// are coalesced; the values of a block go to a few runs (one per window), so
// the stores stay mostly whole sectors.
__global__ void __launch_bounds__(kPermuteBlock) scatter_kernel(const float *src,
                                                               const int32_t *pos, float *dst,
                                                               int64_t nnz)
{
    const int64_t base =
        (int64_t)blockIdx.x * (kPermuteBlock * kPermutePerThread) + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kPermutePerThread; ++j) {
        const int64_t p = base + (int64_t)kPermuteBlock * j;
        if (p < nnz)
            dst[__ldcs(pos + p)] = __ldcs(src + p);
    }
}

cudaError_t launch_values_t(const fmm_plan *p, const float *src, float *dst, cudaStream_t st)
{
    if (p->nnz == 0 || !src)
        return cudaSuccess;
    if (!p->win_pos1)
        return launch_permute(src, p->perm_t, dst, p->nnz, st);
    const int64_t per_block = kPermuteBlock * kPermutePerThread;
    const int64_t blocks = (p->nnz + per_block - 1) / per_block;
    scatter_kernel<<<(unsigned)blocks, kPermuteBlock, 0, st>>>(src, p->win_pos1, p->win_tmp,
                                                              p->nnz);
    permute_kernel<<<(unsigned)blocks, kPermuteBlock, 0, st>>>(p->win_tmp, p->win_pos2, dst,
                                                              p->nnz);
    return cudaGetLastError();
}

__global__ void combine_kernel(const int4 *split, int32_t n_split, const float *partials,
                               float *out, int32_t r, int32_t accumulate)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_split)
        return;
    const int4 sp = split[w];
    for (int k = lane; k < r; k += 32) {
        float acc = 0.f;
        for (int c = 0; c < sp.z; ++c)
            acc += partials[(size_t)(sp.y + c) * r + k];
        out[(size_t)sp.x * r + k] = accumulate ? out[(size_t)sp.x * r + k] + acc : acc;
    }
}

cudaError_t launch_combine(const Side &side, float *out, int32_t r, bool accumulate,
                           cudaStream_t st)
{
    if (side.n_split == 0 || !out)
        return cudaSuccess;
    combine_kernel<<<(side.n_split + 7) / 8, 256, 0, st>>>(side.split, side.n_split,
                                                           side.partials, out, r,
                                                           accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace fmm
