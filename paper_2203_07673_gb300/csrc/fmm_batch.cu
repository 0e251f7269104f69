// Batched FusedMM: many uneven matrices in one persistent launch.
//
// Every matrix of a batch keeps its own plan (pattern, S^T, row order).  A
// batch lists, for each matrix and each row pass of a phase, work units of
// consecutive teams (rows in the plan's longest-first order).  Units of all
// matrices are sorted longest-rows-first and handed out by a device counter:
// every warp of a grid sized to fill the GPU pops a unit, runs the team
// kernel body of that matrix's row width and kernel variant on it, and pops
// the next, until the list is empty.  Forward (FusedMMA of every matrix) is
// one launch; backward (dA and ds over S, dB over S^T, for every matrix) is
// one launch.  The counter is cleared by a memset queued before each launch,
// so both phases can be captured in a CUDA graph and replayed.
//
// Rows are never split in a batch (plans must have no split rows or
// columns): a long row is simply a unit of its own at the head of the list.
// Results are bitwise those of the per-matrix calls with the same variants.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fmm_rows.cuh"

namespace fmm {

struct BatchItemDev {
    PassArgs fwd;       // over S: FusedMMA
    PassArgs bwd_row;   // over S: dA (and ds)
    PassArgs bwd_col;   // over S^T: dB
    int32_t code_fwd;   // (r << 16) | variant code of each role
    int32_t code_row;
    int32_t code_col;
};

enum UnitKind { U_FWD = 0, U_BWD_ROW = 1, U_BWD_COL = 2 };

// Teams [begin, begin + count) of pass `a` (rows order[begin...]).
template <int MODE, typename T, int R, int VPL, int NG, int U>
__device__ __forceinline__ void run_unit(const PassArgs &a, int begin, int count)
{
    constexpr int TEAM = TeamShape<T, R, VPL, NG>::TEAM;
    constexpr int TPW = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    for (int t0 = 0; t0 < count; t0 += TPW) {
        const int t = t0 + lane / TEAM;
        team_pass_body<MODE, T, R, VPL, NG, U>(a, (long long)a.n_chunks + begin + t, t < count);
    }
}

// The variant codes a batch can run: one kernel holds every (width, code)
// path, and its register count is the largest path's, so batches take only
// light variants: at most 32 floats live per lane in the forward phase (64
// registers, 4 blocks per SM; with 48 it needed 80 and ran 19 % slower on
// the 512-matrix batch) and 48 in the backward phase, whose pass over S^T
// holds two gathered rows per nonzero.
template <int MODE, typename T>
constexpr bool batch_code_ok(int r, int code)
{
    const int vecs = r * (int)sizeof(T) / 16;
    const int base = vecs > 32 ? vecs / 32 : 1;
    const int V = (code / 100) * base, N = (code / 10) % 10, UU = code % 10;
    if (V < 1 || vecs % V != 0) return false;
    const int g = vecs / V;
    const int E = V * (16 / (int)sizeof(T));
    const int live = E * (UU * (MODE == M_BWD_COL ? 2 : 1) + 2 + (MODE == M_BWD_ROW ? 1 : 0));
    return g >= 1 && (g & (g - 1)) == 0 && g * N <= 32 && 32 % (g * N) == 0 &&
           live <= (MODE == M_FUSED ? 32 : 48);
}

template <int MODE, typename T>
__device__ __forceinline__ void run_code(int code, const PassArgs &a, int begin, int count)
{
#define FMM_BATCH_CASE(RR, M, N, UU)                                                         \
    case (RR << 16) | (M * 100 + N * 10 + UU):                                               \
        if constexpr (batch_code_ok<MODE, T>(RR, M * 100 + N * 10 + UU))                    \
            run_unit<MODE, T, RR, M * base_vpl<T, RR>(), N, UU>(a, begin, count);            \
        return;
#define FMM_BATCH_R(RR)                                                                      \
    FMM_BATCH_CASE(RR, 1, 1, 2) FMM_BATCH_CASE(RR, 1, 1, 4) FMM_BATCH_CASE(RR, 1, 2, 2)     \
    FMM_BATCH_CASE(RR, 2, 1, 2) FMM_BATCH_CASE(RR, 2, 1, 4) FMM_BATCH_CASE(RR, 2, 2, 1)
    switch (code) {
        FMM_BATCH_R(32)
        FMM_BATCH_R(64)
        FMM_BATCH_R(128)
        FMM_BATCH_R(256)
    default: return;
    }
#undef FMM_BATCH_R
#undef FMM_BATCH_CASE
}

template <typename T, int PHASE>
__global__ void __launch_bounds__(256) batch_kernel(const BatchItemDev *items, const int4 *units,
                                                    int n_units, int *counter)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int u = 0;
        if (lane == 0)
            u = atomicAdd(counter, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units)
            break;
        const int4 unit = units[u];
        const BatchItemDev &it = items[unit.x];
        if constexpr (PHASE == 0) {
            run_code<M_FUSED, T>(it.code_fwd, it.fwd, unit.z, unit.w);
        } else {
            if (unit.y == U_BWD_ROW)
                run_code<M_BWD_ROW, T>(it.code_row, it.bwd_row, unit.z, unit.w);
            else
                run_code<M_BWD_COL, T>(it.code_col, it.bwd_col, unit.z, unit.w);
        }
    }
}

template <typename T>
bool batch_supported(int mode, int r, int code)
{
    switch (mode) {
    case M_FUSED: return batch_code_ok<M_FUSED, T>(r, code);
    case M_BWD_ROW: return batch_code_ok<M_BWD_ROW, T>(r, code);
    default: return batch_code_ok<M_BWD_COL, T>(r, code);
    }
}

// Codes a batch accepts (the FMM_BATCH_R list below).
inline bool batch_listed(int code)
{
    return code == 112 || code == 114 || code == 122 || code == 212 || code == 214 || code == 221;
}

}  // namespace fmm

using namespace fmm;

struct fmm_batch {
    int32_t count = 0, dtype = 0, device = 0;
    bool has_bwd = false;
    BatchItemDev *d_items = nullptr;
    int4 *d_units_fwd = nullptr, *d_units_bwd = nullptr;
    int32_t n_fwd = 0, n_bwd = 0;
    int *d_counters = nullptr;
    int grid_fwd = 0, grid_bwd = 0;
};

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The variant a batch runs for a pass: the plan's, if the batch kernels
// have it for this width and role, else the width's default.
int batch_code(int dtype, int mode, int r, const KernelVariant &v)
{
    const int want = encode_variant(v);
    const bool ok = batch_listed(want) &&
                    (dtype == FMM_BF16 ? batch_supported<bf16_t>(mode, r, want)
                                       : batch_supported<float>(mode, r, want));
    if (ok)
        return want;
    // the default team layout of the width (the batch kernels run the team
    // pass only), with fewer nonzeros per batch if needed
    KernelVariant d = team_default_variant(r, dtype);
    for (int u : {d.u, 2, 1}) {
        d.u = u;
        const int c = encode_variant(d);
        const bool dok = dtype == FMM_BF16 ? batch_supported<bf16_t>(mode, r, c)
                                           : batch_supported<float>(mode, r, c);
        if (dok)
            return c;
    }
    return 112;
}

// Teams per warp of a variant code at width r.
int teams_per_warp(int dtype, int r, int code)
{
    const int vecs = r * (dtype == FMM_BF16 ? 2 : 4) / 16;
    const int base = vecs > 32 ? vecs / 32 : 1;
    const int V = (code / 100) * base, N = (code / 10) % 10;
    return 32 / ((vecs / V) * N);
}

// Units of one pass: consecutive teams within one length bucket, about 512
// nonzeros of work each (from the bucket's shortest row length), a multiple
// of the warp's team count.
void make_units(std::vector<std::pair<int, int4>> &out, const Side &side, int item, int kind,
                int tpw)
{
    for (int key = 0; key < 256; ++key) {
        const int b0 = side.bucket_start[key], b1 = side.bucket_start[key + 1];
        if (b1 <= b0)
            continue;
        int per = tpw;
        if (key >= 136 && key < 255) {
            const int lo = length_key_min((uint32_t)key);
            per = std::max(tpw, std::min(256, 512 / std::max(lo, 1)));
            per = (per + tpw - 1) / tpw * tpw;
        } else if (key == 255) {
            per = 256;                        // empty rows: zero fills
        }
        for (int t = b0; t < b1; t += per)
            out.push_back({key, make_int4(item, kind, t, std::min(per, b1 - t))});
    }
}

int grid_for(const void *kernel)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0);
    return std::max(1, sms * std::max(1, per));
}

#define CHECK(x)              \
    do {                      \
        int _rc = (x);        \
        if (_rc) return _rc;  \
    } while (0)

}  // namespace

extern "C" {

int fmm_plan_set_variant(fmm_plan *p, int32_t variant, int32_t variant_t)
{
    if (!p || (variant && !variant_known(variant)) || (variant_t && !variant_known(variant_t))) {
        set_error_msg("invalid plan or variant code");
        return FMM_EINVAL;
    }
    if (variant)
        p->rows.variant = decode_variant(variant);
    if (variant_t)
        p->cols.variant = decode_variant(variant_t);
    return FMM_OK;
}

int fmm_batch_create(const fmm_batch_item *items, int32_t count, fmm_stream stream,
                     fmm_batch **batch)
{
    if (!batch || !items || count < 1) {
        set_error_msg("fmm_batch_create: NULL argument or empty batch");
        return FMM_EINVAL;
    }
    *batch = nullptr;
    const int dtype = items[0].plan ? items[0].plan->dtype : -1;
    int dev = -1;
    cudaGetDevice(&dev);
    bool bwd = true;
    for (int i = 0; i < count; ++i) {
        const fmm_batch_item &it = items[i];
        const fmm_plan *p = it.plan;
        if (!p || p->dtype != dtype || p->device != dev) {
            set_error_msg("batch items need plans of one dtype on the current device");
            return FMM_EINVAL;
        }
        if (!fast_r(p->r)) {
            set_error_msg("batch items need r in {32, 64, 128, 256}");
            return FMM_EUNSUPPORTED;
        }
        if (p->rows.n_split || (p->has_t && p->cols.n_split)) {
            set_error_msg("batch plans must have no split rows (create them with a large split_nnz)");
            return FMM_EUNSUPPORTED;
        }
        const void *ptrs[] = {it.A, it.B, it.out, it.G, it.dA, it.dB};
        for (const void *q : ptrs)
            if (!aligned16(q)) {
                set_error_msg("batch dense operands must be 16-byte aligned");
                return FMM_EUNSUPPORTED;
            }
        if ((p->m > 0 && (!it.A || !it.out)) || (p->n > 0 && !it.B)) {
            set_error_msg("batch item without A, B or out");
            return FMM_EINVAL;
        }
        if (!it.G || (!it.dA && !it.dB && !it.ds) || (it.dB && !p->has_t))
            bwd = false;
    }
    std::vector<BatchItemDev> host(count);
    std::vector<std::pair<int, int4>> uf, ub;
    for (int i = 0; i < count; ++i) {
        const fmm_batch_item &it = items[i];
        const fmm_plan *p = it.plan;
        BatchItemDev &d = host[i];
        auto fill = [&](PassArgs &a, const Side &side, const float *s, const void *L,
                        const void *Y, const float *H, float *out, float *nzout) {
            a.row_ptr = side.row_ptr;
            a.col_idx = side.col_idx;
            a.perm = side.perm;
            a.order = side.light_order();
            a.n_light = side.n_light;
            a.chunks = nullptr;
            a.n_chunks = 0;
            a.partials = nullptr;
            a.s = s;
            a.s_direct = 0;
            a.L = L;
            a.Y = Y;
            a.H = H;
            a.out = out;
            a.nzout = nzout;
            a.r = p->r;
        };
        fill(d.fwd, p->rows, it.vals, it.A, it.B, nullptr, it.out, nullptr);
        fill(d.bwd_row, p->rows, it.vals, it.A, it.B, it.G, it.dA, it.ds);
        PassArgs empty{};
        d.bwd_col = empty;
        if (p->has_t)
            fill(d.bwd_col, p->cols, it.vals, it.B, it.A, it.G, it.dB, nullptr);
        const int cf = batch_code(dtype, M_FUSED, p->r, p->rows.variant);
        d.code_fwd = (p->r << 16) | cf;
        make_units(uf, p->rows, i, U_FWD, teams_per_warp(dtype, p->r, cf));
        d.code_row = d.code_col = 0;
        if (bwd) {
            const int cr = batch_code(dtype, M_BWD_ROW, p->r, p->rows.variant);
            d.code_row = (p->r << 16) | cr;
            if (it.dA || it.ds)
                make_units(ub, p->rows, i, U_BWD_ROW, teams_per_warp(dtype, p->r, cr));
            if (it.dB) {
                const int cc = batch_code(dtype, M_BWD_COL, p->r, p->cols.variant);
                d.code_col = (p->r << 16) | cc;
                make_units(ub, p->cols, i, U_BWD_COL, teams_per_warp(dtype, p->r, cc));
            }
        }
    }
    auto by_key = [](const std::pair<int, int4> &x, const std::pair<int, int4> &y) {
        return x.first < y.first;
    };
    std::stable_sort(uf.begin(), uf.end(), by_key);
    std::stable_sort(ub.begin(), ub.end(), by_key);
    fmm_batch *b = new fmm_batch();
    b->count = count;
    b->dtype = dtype;
    b->device = dev;
    b->has_bwd = bwd;
    b->n_fwd = (int32_t)uf.size();
    b->n_bwd = (int32_t)ub.size();
    std::vector<int4> units_f(uf.size()), units_b(ub.size());
    for (size_t k = 0; k < uf.size(); ++k) units_f[k] = uf[k].second;
    for (size_t k = 0; k < ub.size(); ++k) units_b[k] = ub[k].second;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BatchItemDev) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_units_fwd, sizeof(int4) * std::max<size_t>(1, uf.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_units_bwd, sizeof(int4) * std::max<size_t>(1, ub.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, host.data(), sizeof(BatchItemDev) * count,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !uf.empty())
        e = cudaMemcpyAsync(b->d_units_fwd, units_f.data(), sizeof(int4) * uf.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ub.empty())
        e = cudaMemcpyAsync(b->d_units_bwd, units_b.data(), sizeof(int4) * ub.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("fmm_batch_create", e);
        fmm_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA;
    }
    if (dtype == FMM_BF16) {
        b->grid_fwd = grid_for((const void *)batch_kernel<bf16_t, 0>);
        b->grid_bwd = grid_for((const void *)batch_kernel<bf16_t, 1>);
    } else {
        b->grid_fwd = grid_for((const void *)batch_kernel<float, 0>);
        b->grid_bwd = grid_for((const void *)batch_kernel<float, 1>);
    }
    *batch = b;
    return FMM_OK;
}

int fmm_batch_forward(const fmm_batch *b, fmm_stream stream)
{
    if (!b) {
        set_error_msg("batch is NULL");
        return FMM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int), st);
    if (e == cudaSuccess && b->n_fwd > 0) {
        if (b->dtype == FMM_BF16)
            batch_kernel<bf16_t, 0><<<b->grid_fwd, 256, 0, st>>>(b->d_items, b->d_units_fwd,
                                                                 b->n_fwd, b->d_counters);
        else
            batch_kernel<float, 0><<<b->grid_fwd, 256, 0, st>>>(b->d_items, b->d_units_fwd,
                                                                b->n_fwd, b->d_counters);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fmm_batch_forward", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

int fmm_batch_backward(const fmm_batch *b, fmm_stream stream)
{
    if (!b) {
        set_error_msg("batch is NULL");
        return FMM_EINVAL;
    }
    if (!b->has_bwd) {
        set_error_msg("batch built without G and gradient outputs (or without S^T)");
        return FMM_EUNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(b->d_counters + 1, 0, sizeof(int), st);
    if (e == cudaSuccess && b->n_bwd > 0) {
        if (b->dtype == FMM_BF16)
            batch_kernel<bf16_t, 1><<<b->grid_bwd, 256, 0, st>>>(b->d_items, b->d_units_bwd,
                                                                 b->n_bwd, b->d_counters + 1);
        else
            batch_kernel<float, 1><<<b->grid_bwd, 256, 0, st>>>(b->d_items, b->d_units_bwd,
                                                                b->n_bwd, b->d_counters + 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fmm_batch_backward", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

int fmm_batch_destroy(fmm_batch *b)
{
    if (!b)
        return FMM_OK;
    cudaDeviceSynchronize();
    cudaFree(b->d_items);
    cudaFree(b->d_units_fwd);
    cudaFree(b->d_units_bwd);
    cudaFree(b->d_counters);
    delete b;
    return FMM_OK;
}

}  // extern "C"
