// Graph-attention layer, forward (Sec. VI-E): the attention variant of SDDMM
// feeding a softmax-normalised SpMM, one gather pass per row.
//
// One head scores the nonzero (i, j) with e_ij = LeakyReLU(s_ij (f_i + g_j)),
// where f = H a_l and g = H a_r are per-node projections (the a^T (H_i || H_j)
// of the paper's GAT product), normalises the scores of row i with a softmax
// and aggregates out_i = sum_j softmax(e)_ij H_j.  With per-node projections
// the sampled "dot product" of an edge is one addition, so the pass is a
// gather of H_j (and the scalar g_j) per nonzero.  The softmax is computed
// online: each lane holds 8 consecutive elements of the row, all in one head
// (the head width is a multiple of 8), and keeps that head's running
// maximum, the running sum of exp(e - max) and its exp-weighted accumulator,
// rescaled when the maximum grows; no cross-lane reduction is needed.  Rows
// without nonzeros give zeros.  Long rows are processed in the
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

// Eight consecutive elements of a row, widened to float: one 32-byte load of
// float32 or one 16-byte load of bfloat16 (the read-only path for gathered
// rows).  p must be 32-byte (float) or 16-byte (bfloat16) aligned.
__device__ __forceinline__ void load8(const float *p, float *f)
{
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]),
                   "=f"(f[6]), "=f"(f[7])
                 : "l"(p));
}
__device__ __forceinline__ void load8(const bf16_t *p, float *f)
{
    unpack_bf16x8(__ldg(reinterpret_cast<const uint4 *>(p)), f);
}
// Eight floats to a 16-byte-aligned address, streaming (written once).
__device__ __forceinline__ void store8(float *p, const float *f)
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(f[0], f[1], f[2], f[3]));
    __stcs(reinterpret_cast<float4 *>(p) + 1, make_float4(f[4], f[5], f[6], f[7]));
}

// One row (or chunk) per team of G = R / 8 lanes; lane l holds elements
// [8 l, 8 l + 8) of the row, all in head 8 l / rh (rh a multiple of 8), so a
// lane scores each nonzero once for its head.  Online softmax per lane:
// with d = e - max, exactly one of exp(max_old - max_new) and exp(e - max_new)
// differs from 1, so one exponential x = exp(-|d|) gives both; when the score
// does not raise the maximum (the common case, uniform across a head's lanes)
// the update is acc += x H_j, else acc = x acc + H_j.  U nonzeros per batch,
// their gathers in flight together.  Capped at 48 registers (5 blocks per
// SM): 17-20 % faster on GB300 than the uncapped 58.
template <typename T, int R, int U>
__global__ void __launch_bounds__(256, 5) gat_kernel(const GatArgs a)
{
    constexpr int G = R / 8;
    static_assert(R % 8 == 0 && G >= 1 && G <= 32 && (G & (G - 1)) == 0, "row layout");
    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long total = (long long)a.n_chunks + a.n_light;
    const bool active = gid < total;
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
    const int head = (8 * lig) / a.rh;
    const float *g = a.g + head;
    const float fi = active && end > beg ? __ldg(a.f + (size_t)row * a.heads + head) : 0.f;
    float mx = -INFINITY, l = 0.f, acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;

    // The team loads the column indices and values of IB >= 16 consecutive
    // nonzeros at once (K per lane, coalesced) and hands them to its batches
    // by shuffles, so the index latency is paid once per IB / U batches.
    constexpr int K = G >= 16 ? 1 : 16 / G;
    constexpr int IB = K * G;
    static_assert(IB % U == 0, "whole batches per index block");
    const int tbase = lane & ~(G - 1);
    const int blocks = (end - beg + IB - 1) / IB;
    const int wblocks = (int)__reduce_max_sync(0xffffffffu, (unsigned)blocks);
    for (int bk = 0; bk < wblocks; ++bk) {
        int mj[K];
        float ms[K];
#pragma unroll
        for (int e = 0; e < K; ++e) {
            const int p = beg + bk * IB + e * G + lig;
            mj[e] = p < end ? __ldg(a.col_idx + p) : -1;
            ms[e] = (p < end && a.s) ? __ldg(a.s + p) : 1.f;
        }
#pragma unroll 1
        for (int sub = 0; sub < IB / U; ++sub) {
            int jj[U];
            float sv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int o = sub * U + u;
                const int e = o / G, src = tbase + o % G;
                int jv = mj[0];
                float svv = ms[0];
#pragma unroll
                for (int t = 1; t < K; ++t)
                    if (e == t) { jv = mj[t]; svv = ms[t]; }
                jj[u] = __shfl_sync(0xffffffffu, jv, src);
                sv[u] = __shfl_sync(0xffffffffu, svv, src);
            }
            float y[U][8], gj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] >= 0) {
                    load8(H + (size_t)jj[u] * R + 8 * lig, y[u]);
                    gj[u] = __ldg(g + (size_t)jj[u] * a.heads);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] < 0)
                    continue;
                const float e = leaky(sv[u] * (fi + gj[u]), a.slope);
                const float d = e - mx;                 // +inf for the first nonzero
                const float x = __expf(-fabsf(d));      // 0 for the first nonzero
                if (d > 0.f) {
                    l = fmaf(l, x, 1.f);
#pragma unroll
                    for (int t = 0; t < 8; ++t) acc[t] = fmaf(acc[t], x, y[u][t]);
                    mx = e;
                } else {
                    l += x;
#pragma unroll
                    for (int t = 0; t < 8; ++t) acc[t] = fmaf(x, y[u][t], acc[t]);
                }
            }
        }
    }
    if (!active)
        return;
    if (slot >= 0) {
        // a chunk: keep the unnormalised state for the combine kernel
        float *base = a.partials + (size_t)slot * 3 * R + 8 * lig;
        float mxe[8], le[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) { mxe[t] = mx; le[t] = l; }
        store8(base, acc);
        store8(base + R, mxe);
        store8(base + 2 * R, le);
    } else {
        const float inv = l > 0.f ? 1.f / l : 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] *= inv;
        store8(a.out + (size_t)row * R + 8 * lig, acc);
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

template <typename T, int R, int U>
cudaError_t launch_gat_vec(const GatArgs &a, cudaStream_t st)
{
    constexpr int G = R / 8;
    const long long total = (long long)a.n_chunks + a.n_light;
    gat_kernel<T, R, U><<<(unsigned)((total * G + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Vector path: 8 elements per lane, 2 nonzeros per batch.
template <typename T>
cudaError_t launch_gat(const GatArgs &a, bool vec, cudaStream_t st)
{
    const long long total = (long long)a.n_chunks + a.n_light;
    if (total == 0)
        return cudaSuccess;
    if (vec && a.rh % 8 == 0) {
        switch (a.r) {
        case 32: return launch_gat_vec<T, 32, 2>(a, st);
        case 64: return launch_gat_vec<T, 64, 2>(a, st);
        case 128: return launch_gat_vec<T, 128, 2>(a, st);
        case 256: return launch_gat_vec<T, 256, 2>(a, st);
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
    const int64_t blocks = std::min<int64_t>(((int64_t)rows + 7) / 8, (int64_t)sm_count() * 64);
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
    // the vector path loads 8 elements of H per lane (32 bytes of float32 or
    // 16 bytes of bfloat16) and stores 16-byte halves of out
    const uintptr_t h_align = p->dtype == FMM_BF16 ? 15u : 31u;
    const bool vec = fast_r(p->r) && (reinterpret_cast<uintptr_t>(H) & h_align) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
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
