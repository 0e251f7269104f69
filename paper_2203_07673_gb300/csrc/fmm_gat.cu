// Graph-attention layer, forward (Sec. VI-E): the attention variant of SDDMM
// feeding a softmax-normalised SpMM, one gather pass per row.
//
// One head scores the nonzero (i, j) with e_ij = LeakyReLU(s_ij (f_i + g_j)),
// where f = H a_l and g = H a_r are per-node projections (the a^T (H_i || H_j)
// of the paper's GAT product), normalises the scores of row i with a softmax
// and aggregates out_i = sum_j softmax(e)_ij H_j.  With per-node projections
// the sampled "dot product" of an edge is one addition, so the pass is a
// gather of H_j (and the scalar g_j) per nonzero.  The softmax is computed
// online: each lane keeps, per 16-byte vector of the row it holds (a vector
// lies in one head when the head width is a multiple of its element count),
// the running maximum, the running sum of exp(e - max) and the exp-weighted
// accumulator, rescaled when the maximum grows; no cross-lane reduction is
// needed.  Rows without nonzeros give zeros.  Long rows are processed in the
// plan's chunks: every chunk leaves its accumulator, maximum and sum per
// element in the plan's partials, and a combine kernel merges the chunks of
// a row in chunk order (max of the maxima, sums rescaled to it): results
// stay deterministic.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "fmm_rows.cuh"

namespace fmm {

struct GatArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *order;     // light rows
    int32_t n_light;
    const int4 *chunks;       // chunks of split rows (row, begin, end)
    int32_t n_chunks;
    float *partials;          // per chunk: acc (r), max (r), sum (r)
    const int4 *split;        // split rows (row, first chunk, chunk count)
    int32_t n_split;
    const float *s;           // values (NULL = 1)
    const float *f;           // m x heads
    const float *g;           // n x heads
    const void *H;            // n x r
    float *out;               // m x r
    int32_t heads, rh, r;
    float slope;
};

__device__ __forceinline__ float leaky(float x, float slope) { return x > 0.f ? x : slope * x; }

template <typename T, int R, int VPL, int U>
__global__ void __launch_bounds__(256) gat_kernel(const GatArgs a)
{
    using TS = TeamShape<T, R, VPL, 1>;
    constexpr int G = TS::G, E = TS::E, EPV = TS::EPV;
    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long total = (long long)a.n_chunks + a.n_light;
    const bool active = gid < total;
    const Loader ld;
    int row = 0, beg = 0, end = 0, slot = -1;
    if (active) {
        if (gid < a.n_chunks) {
            const int4 c = a.chunks[gid];
            row = c.x; beg = c.y; end = c.z; slot = (int)gid;
        } else {
            row = a.order[gid - a.n_chunks];
            beg = __ldg(a.row_ptr + row);
            end = __ldg(a.row_ptr + row + 1);
        }
    }
    const T *H = static_cast<const T *>(a.H);
    int head[VPL];
    float fi[VPL], mx[VPL], l[VPL], acc[E];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        head[v] = ((v * G + lig) * EPV) / a.rh;
        fi[v] = active && end > beg ? __ldg(a.f + (size_t)row * a.heads + head[v]) : 0.f;
        mx[v] = -INFINITY;
        l[v] = 0.f;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = 0.f;

    const int iters = (end - beg + U - 1) / U;
    const int witers = (int)__reduce_max_sync(0xffffffffu, (unsigned)iters);
    for (int it = 0; it < witers; ++it) {
        int jj[U];
        float sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = beg + it * U + u;
            jj[u] = p < end ? __ldg(a.col_idx + p) : -1;
            sv[u] = (p < end && a.s) ? __ldg(a.s + p) : 1.f;
        }
        float y[U][E], gj[U][VPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                team_load<T, VPL, G>(ld, H + (size_t)jj[u] * R, lig, y[u], true);
#pragma unroll
                for (int v = 0; v < VPL; ++v)
                    gj[u][v] = __ldg(a.g + (size_t)jj[u] * a.heads + head[v]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0)
                continue;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const float e = leaky(sv[u] * (fi[v] + gj[u][v]), a.slope);
                const float mnew = fmaxf(mx[v], e);
                const float c_old = expf(mx[v] - mnew);   // 0 for the first nonzero
                const float c_new = expf(e - mnew);
                l[v] = fmaf(l[v], c_old, c_new);
#pragma unroll
                for (int t = 0; t < EPV; ++t)
                    acc[v * EPV + t] = fmaf(acc[v * EPV + t], c_old, c_new * y[u][v * EPV + t]);
                mx[v] = mnew;
            }
        }
    }
    if (active && slot >= 0) {
        // a chunk: keep the unnormalised state for the combine kernel
        float *base = a.partials + (size_t)slot * 3 * R;
        float mxe[E], le[E];
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int t = 0; t < EPV; ++t) {
                mxe[v * EPV + t] = mx[v];
                le[v * EPV + t] = l[v];
            }
        team_store_f32<T, VPL, G>(ld, base, lig, acc);
        team_store_f32<T, VPL, G>(ld, base + R, lig, mxe);
        team_store_f32<T, VPL, G>(ld, base + 2 * R, lig, le);
    } else if (active) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const float inv = l[v] > 0.f ? 1.f / l[v] : 0.f;
#pragma unroll
            for (int t = 0; t < EPV; ++t)
                acc[v * EPV + t] *= inv;
        }
        team_store_f32<T, VPL, G>(ld, a.out + (size_t)row * R, lig, acc);
    }
}

// Merges the chunk states of every split row, in chunk order:
// M = max_c max_c[k], out[k] = sum_c acc_c[k] e^(max_c[k] - M) /
// sum_c sum_c[k] e^(max_c[k] - M).  One warp per split row.
__global__ void __launch_bounds__(256) gat_combine_kernel(const GatArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= a.n_split)
        return;
    const int4 sp = a.split[w];
    const int r = a.r;
    for (int k = lane; k < r; k += 32) {
        float M = -INFINITY;
        for (int c = 0; c < sp.z; ++c)
            M = fmaxf(M, a.partials[(size_t)(sp.y + c) * 3 * r + r + k]);
        float A = 0.f, L = 0.f;
        if (M > -INFINITY) {
            for (int c = 0; c < sp.z; ++c) {
                const float *b = a.partials + (size_t)(sp.y + c) * 3 * r;
                const float wgt = expf(b[r + k] - M);
                A = fmaf(b[k], wgt, A);
                L = fmaf(b[2 * r + k], wgt, L);
            }
        }
        a.out[(size_t)sp.x * r + k] = L > 0.f ? A / L : 0.f;
    }
}

// Any width: one warp per row, one pass over the row's nonzeros per head.
template <typename T>
__global__ void __launch_bounds__(256) gat_generic(const GatArgs a)
{
    const int lane = threadIdx.x & 31;
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long total = (long long)a.n_chunks + a.n_light;
    if (gid >= total)
        return;
    int row, beg, end, slot = -1;
    if (gid < a.n_chunks) {
        const int4 c = a.chunks[gid];
        row = c.x; beg = c.y; end = c.z; slot = (int)gid;
    } else {
        row = a.order[gid - a.n_chunks];
        beg = __ldg(a.row_ptr + row);
        end = __ldg(a.row_ptr + row + 1);
    }
    const T *H = static_cast<const T *>(a.H);
    // a chunk accumulates into its partial row, a whole row into out
    float *o = slot >= 0 ? a.partials + (size_t)slot * 3 * a.r : a.out + (size_t)row * a.r;
    for (int h = 0; h < a.heads; ++h) {
        const float fi = end > beg ? __ldg(a.f + (size_t)row * a.heads + h) : 0.f;
        float mx = -INFINITY, l = 0.f;
        for (int k = lane; k < a.rh; k += 32)
            o[h * a.rh + k] = 0.f;
        for (int p = beg; p < end; ++p) {
            const int j = __ldg(a.col_idx + p);
            const float sv = a.s ? __ldg(a.s + p) : 1.f;
            const float e = leaky(sv * (fi + __ldg(a.g + (size_t)j * a.heads + h)), a.slope);
            const float mnew = fmaxf(mx, e);
            const float c_old = expf(mx - mnew), c_new = expf(e - mnew);
            l = fmaf(l, c_old, c_new);
            const T *hj = H + (size_t)j * a.r + h * a.rh;
            for (int k = lane; k < a.rh; k += 32)
                o[h * a.rh + k] = fmaf(o[h * a.rh + k], c_old, c_new * widen<T>(hj[k]));
            mx = mnew;
        }
        if (slot >= 0) {
            for (int k = lane; k < a.rh; k += 32) {
                o[a.r + h * a.rh + k] = mx;
                o[2 * a.r + h * a.rh + k] = l;
            }
        } else {
            const float inv = l > 0.f ? 1.f / l : 0.f;
            for (int k = lane; k < a.rh; k += 32)
                o[h * a.rh + k] *= inv;
        }
    }
}

// out[i, h] = sum_k X[i, h*rh + k] * w[h*rh + k]: the per-node projections
// f = H a_l and g = H a_r of every head.  One warp per row.
__global__ void __launch_bounds__(256) gat_project_kernel(int32_t rows, int32_t heads, int32_t rh,
                                                          const float *X, const float *w,
                                                          float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int r = heads * rh;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += warps) {
        for (int h = 0; h < heads; ++h) {
            float acc = 0.f;
            for (int k = lane; k < rh; k += 32)
                acc = fmaf(X[(size_t)i * r + h * rh + k], w[h * rh + k], acc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0)
                out[(size_t)i * heads + h] = acc;
        }
    }
}

template <typename T, int R, int VPL, int U>
cudaError_t launch_gat_vec(const GatArgs &a, cudaStream_t st)
{
    constexpr int G = TeamShape<T, R, VPL, 1>::G;
    const long long total = (long long)a.n_chunks + a.n_light;
    gat_kernel<T, R, VPL, U><<<(unsigned)((total * G + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Vector path: 8 elements per lane (as the default variant of the row
// passes), 2 nonzeros per batch.
template <typename T>
cudaError_t launch_gat(const GatArgs &a, bool vec, cudaStream_t st)
{
    const long long total = (long long)a.n_chunks + a.n_light;
    if (total == 0)
        return cudaSuccess;
    constexpr int EPV = 16 / (int)sizeof(T);
    if (vec && a.rh % EPV == 0) {
        constexpr int V1 = sizeof(T) == 4 ? 2 : 1;   // vectors per lane for 8 elements
        switch (a.r) {
        case 32: return launch_gat_vec<T, 32, V1, 2>(a, st);
        case 64: return launch_gat_vec<T, 64, V1, 2>(a, st);
        case 128: return launch_gat_vec<T, 128, V1, 2>(a, st);
        case 256: return launch_gat_vec<T, 256, (sizeof(T) == 4 ? 2 : 1), 2>(a, st);
        default: break;
        }
    }
    gat_generic<T><<<(unsigned)((total + 7) / 8), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fmm

using namespace fmm;

extern "C" {

int fmm_gat_project(int32_t rows, int32_t heads, int32_t rh, const float *X, const float *w,
                    float *out, fmm_stream stream)
{
    if (rows < 0 || heads < 1 || rh < 1 || (rows > 0 && (!X || !w || !out))) {
        set_error_msg("fmm_gat_project: invalid arguments");
        return FMM_EINVAL;
    }
    if (rows == 0)
        return FMM_OK;
    const int64_t blocks = std::min<int64_t>(((int64_t)rows + 7) / 8, 152 * 64);
    gat_project_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(rows, heads, rh, X, w,
                                                                          out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("fmm_gat_project", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

int fmm_gat_forward(const fmm_plan *p, int32_t heads, const float *vals, const float *f,
                    const float *g, const void *H, float slope, float *out, fmm_stream stream)
{
    if (!p) {
        set_error_msg("plan is NULL");
        return FMM_EINVAL;
    }
    if (heads < 1 || p->r % heads != 0) {
        set_error_msg("fmm_gat_forward: heads must divide r");
        return FMM_EINVAL;
    }
    if ((p->m > 0 && (!f || !out)) || (p->n > 0 && (!g || !H))) {
        set_error_msg("fmm_gat_forward: NULL operand");
        return FMM_EINVAL;
    }
    GatArgs a;
    a.row_ptr = p->rows.row_ptr;
    a.col_idx = p->rows.col_idx;
    a.order = p->rows.light_order();
    a.n_light = p->rows.n_light;
    a.chunks = p->rows.chunks;
    a.n_chunks = p->rows.n_chunks;
    a.partials = p->rows.partials;
    a.split = p->rows.split;
    a.n_split = p->rows.n_split;
    a.s = vals;
    a.f = f;
    a.g = g;
    a.H = H;
    a.out = out;
    a.heads = heads;
    a.rh = p->r / heads;
    a.r = p->r;
    a.slope = slope;
    const bool vec = fast_r(p->r) && ((reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = p->dtype == FMM_BF16 ? launch_gat<bf16_t>(a, vec, st)
                                         : launch_gat<float>(a, vec, st);
    if (e == cudaSuccess && a.n_split > 0) {
        gat_combine_kernel<<<(a.n_split + 7) / 8, 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("fmm_gat_forward", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

}  // extern "C"
