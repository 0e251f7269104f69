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

// EPL consecutive elements of a gathered row as loaded (EPL a multiple of
// 8): float32 rows in registers as floats (32-byte loads), bfloat16 rows kept
// packed two to a word until use, so a nonzero in flight costs EPL / 2
// registers (16-byte loads for EPL = 8, 32-byte loads for EPL = 16).  The
// read-only path; the address must be aligned to the load width.
template <typename T, int EPL>
struct GatRaw;

template <int EPL>
struct GatRaw<float, EPL> {
    float v[EPL];
    __device__ __forceinline__ void load(const float *p)
    {
#pragma unroll
        for (int k = 0; k < EPL / 8; ++k)
            asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=f"(v[8 * k]), "=f"(v[8 * k + 1]), "=f"(v[8 * k + 2]),
                           "=f"(v[8 * k + 3]), "=f"(v[8 * k + 4]), "=f"(v[8 * k + 5]),
                           "=f"(v[8 * k + 6]), "=f"(v[8 * k + 7])
                         : "l"(p + 8 * k));
    }
    __device__ __forceinline__ float get(int t) const { return v[t]; }
};

template <int EPL>
struct GatRaw<bf16_t, EPL> {
    uint32_t w[EPL / 2];
    __device__ __forceinline__ void load(const bf16_t *p)
    {
        if constexpr (EPL % 16 == 0) {
#pragma unroll
            for (int k = 0; k < EPL / 16; ++k)
                asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(w[8 * k]), "=r"(w[8 * k + 1]), "=r"(w[8 * k + 2]),
                               "=r"(w[8 * k + 3]), "=r"(w[8 * k + 4]), "=r"(w[8 * k + 5]),
                               "=r"(w[8 * k + 6]), "=r"(w[8 * k + 7])
                             : "l"(p + 16 * k));
        } else {
#pragma unroll
            for (int k = 0; k < EPL / 8; ++k) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p + 8 * k));
                w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
            }
        }
    }
    // element t: the low half of word t / 2 for even t, the high half for odd
    __device__ __forceinline__ float get(int t) const
    {
        return (t & 1) ? __uint_as_float(w[t >> 1] & 0xffff0000u) : __uint_as_float(w[t >> 1] << 16);
    }
};

// Eight floats to a 16-byte-aligned address, streaming (written once).
__device__ __forceinline__ void store8(float *p, const float *f)
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(f[0], f[1], f[2], f[3]));
    __stcs(reinterpret_cast<float4 *>(p) + 1, make_float4(f[4], f[5], f[6], f[7]));
}

// Launch shape of the vector path per element type: EPL elements per lane,
// U nonzeros in flight per batch, MINB blocks of 256 threads per SM (the
// register cap).  Measured on GB300 (GAT forward, R-MAT 2^22, 4 heads x 32):
// 16 elements per lane, one nonzero per batch, beat 8 per lane with two
// (float32 3.39 against 3.65 ms, bfloat16 2.62 against 3.18 ms); heads whose
// width is a multiple of 8 but not of 16 take the 8-per-lane shape.
template <typename T>
struct GatConfig;
template <>
struct GatConfig<float> {
    static constexpr int EPL = 16, U = 1, MINB = 3;
};
template <>
struct GatConfig<bf16_t> {
    static constexpr int EPL = 16, U = 1, MINB = 5;
};
struct GatNarrow {
    static constexpr int EPL = 8, U = 2, MINB = 5;
};

// One row (or chunk) per team of G = R / EPL lanes; lane l holds elements
// [EPL l, EPL l + EPL) of the row, all in head EPL l / rh (rh a multiple of
// EPL), so a lane scores each nonzero once for its head.  Online softmax per
// lane: with d = e - max, exactly one of exp(max_old - max_new) and
// exp(e - max_new) differs from 1, so one exponential x = exp(-|d|) gives
// both; when the score does not raise the maximum (the common case, uniform
// across a head's lanes) the update is acc += x H_j, else acc = x acc + H_j.
// U nonzeros per batch, their gathers in flight together.
// Blocks of two warps, MINB blocks of 256 threads' worth resident per SM (a
// register cap of 65536 / (256 MINB)): small blocks retire as soon as their
// rows are done (GB300, R-MAT 2^22, 4 x 32: FP32 H 3.364 -> 3.233 ms, BF16
// H 2.621 -> 2.538 ms against 256-thread blocks).
constexpr int kGatBlock = 64;

template <typename T, int R, int U, int EPL, int MINB>
__global__ void __launch_bounds__(kGatBlock, MINB * (256 / kGatBlock)) gat_kernel(const GatArgs a)
{
    constexpr int G = R / EPL;
    static_assert(EPL % 8 == 0 && R % EPL == 0 && G >= 1 && G <= 32 && (G & (G - 1)) == 0,
                  "row layout");
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
    const int head = (EPL * lig) / a.rh;
    const float *g = a.g + head;
    const float fi = active && end > beg ? __ldg(a.f + (size_t)row * a.heads + head) : 0.f;
    float mx = -INFINITY, l = 0.f, acc[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) acc[e] = 0.f;

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
            GatRaw<T, EPL> y[U];
            float gj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] >= 0) {
                    y[u].load(H + (size_t)jj[u] * R + EPL * lig);
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
                    for (int t = 0; t < EPL; ++t) acc[t] = fmaf(acc[t], x, y[u].get(t));
                    mx = e;
                } else {
                    l += x;
#pragma unroll
                    for (int t = 0; t < EPL; ++t) acc[t] = fmaf(x, y[u].get(t), acc[t]);
                }
            }
        }
    }
    if (!active)
        return;
    if (slot >= 0) {
        // a chunk: keep the unnormalised state for the combine kernel
        float *base = a.partials + (size_t)slot * 3 * R + EPL * lig;
        float mxe[8], le[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) { mxe[t] = mx; le[t] = l; }
#pragma unroll
        for (int k = 0; k < EPL / 8; ++k) {
            store8(base + 8 * k, acc + 8 * k);
            store8(base + R + 8 * k, mxe);
            store8(base + 2 * R + 8 * k, le);
        }
    } else {
        const float inv = l > 0.f ? 1.f / l : 0.f;
#pragma unroll
        for (int t = 0; t < EPL; ++t) acc[t] *= inv;
#pragma unroll
        for (int k = 0; k < EPL / 8; ++k)
            store8(a.out + (size_t)row * R + EPL * lig + 8 * k, acc + 8 * k);
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

template <typename T, int R, typename C>
cudaError_t launch_gat_vec(const GatArgs &a, cudaStream_t st)
{
    constexpr int G = R / C::EPL;
    const long long total = (long long)a.n_chunks + a.n_light;
    gat_kernel<T, R, C::U, C::EPL, C::MINB>
        <<<(unsigned)((total * G + kGatBlock - 1) / kGatBlock), kGatBlock, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_gat_shape(const GatArgs &a, cudaStream_t st)
{
    switch (a.r) {
    case 32: return launch_gat_vec<T, 32, C>(a, st);
    case 64: return launch_gat_vec<T, 64, C>(a, st);
    case 128: return launch_gat_vec<T, 128, C>(a, st);
    default: return launch_gat_vec<T, 256, C>(a, st);
    }
}

// Vector path (r in {32, 64, 128, 256}, out 16-byte aligned):
// GatConfig<T>::EPL elements per lane when the head width is a multiple of
// it and H is 32-byte aligned, else 8 per lane when the head width is a
// multiple of 8 and H is aligned to that shape's loads (32 bytes of float32,
// 16 of bfloat16); otherwise one warp per row.
template <typename T>
cudaError_t launch_gat(const GatArgs &a, bool vec, cudaStream_t st)
{
    const long long total = (long long)a.n_chunks + a.n_light;
    if (total == 0)
        return cudaSuccess;
    const uintptr_t h = reinterpret_cast<uintptr_t>(a.H);
    const bool width = a.r == 32 || a.r == 64 || a.r == 128 || a.r == 256;
    if (vec && width && a.rh % GatConfig<T>::EPL == 0 && (h & 31u) == 0)
        return launch_gat_shape<T, GatConfig<T>>(a, st);
    const uintptr_t narrow_align = sizeof(T) == 2 ? 15u : 31u;
    if (vec && width && a.rh % GatNarrow::EPL == 0 && (h & narrow_align) == 0)
        return launch_gat_shape<T, GatNarrow>(a, st);
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
    // the vector path stores 16-byte pieces of out; launch_gat checks the
    // alignment of H against the loads of the shape it picks
    const bool vec = fast_r(p->r) && (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
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
