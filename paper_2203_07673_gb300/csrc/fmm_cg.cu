// Row-wise conjugate gradients for ALS (Sec. VI-E).
//
// ALS solves, for every row x_i of the factor being updated, the normal
// equations M_i x_i = b_i with M_i x = sum_j <x, Y_j> Y_j + lambda x.  CG
// runs on all rows at once: the product M p of every row is one FusedMM over
// the 0/1 pattern (computed by the caller with fmm_fusedmm or
// fmm_fusedmm_t), and everything else is per-row vector work.  The paper
// found those per-row dot products to be its bottleneck (short vectors, one
// call each); here each CG step's vector work -- two dot products and three
// updates per row -- is one kernel with one warp per row, every row vector
// read and written once.
#include <algorithm>
#include <cstdio>

#include "fmm_internal.cuh"

namespace fmm {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// res = b - mx - lambda x;  p = res;  rs = <res, res>   (row-wise)
// EPL elements per lane: r <= 32 * EPL (lane l holds k = l + 32 t).
template <int EPL>
__global__ void __launch_bounds__(256) cg_init_kernel(int32_t rows, int32_t r, float lambda,
                                                      const float *b, const float *mx,
                                                      const float *x, float *res, float *p,
                                                      float *rs)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
         row += warps) {
        const size_t base = (size_t)row * r;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < EPL; ++t) {
            const int k = lane + 32 * t;
            if (k < r) {
                const float v = b[base + k] - mx[base + k] - lambda * x[base + k];
                res[base + k] = v;
                p[base + k] = v;
                acc = fmaf(v, v, acc);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0)
            rs[row] = acc;
    }
}

// One CG step per row, with q = (M - lambda I) p given:
//   t = q + lambda p;  alpha = rs / <p, t>  (0 if <p, t> <= 0)
//   x += alpha p;  res -= alpha t;  rs' = <res, res>
//   beta = rs' / rs  (0 if rs = 0);  p = res + beta p;  rs = rs'
template <int EPL>
__global__ void __launch_bounds__(256) cg_update_kernel(int32_t rows, int32_t r, float lambda,
                                                        float *x, float *res, float *p,
                                                        const float *q, float *rs)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
         row += warps) {
        const size_t base = (size_t)row * r;
        float pv[EPL], tv[EPL], rv[EPL];
        float pq = 0.f;
#pragma unroll
        for (int t = 0; t < EPL; ++t) {
            const int k = lane + 32 * t;
            pv[t] = 0.f; tv[t] = 0.f; rv[t] = 0.f;
            if (k < r) {
                pv[t] = p[base + k];
                tv[t] = fmaf(lambda, pv[t], q[base + k]);
                rv[t] = res[base + k];
            }
            pq = fmaf(pv[t], tv[t], pq);
        }
        pq = warp_sum(pq);
        const float rs_old = rs[row];
        const float alpha = pq > 0.f ? rs_old / pq : 0.f;
        float rr = 0.f;
#pragma unroll
        for (int t = 0; t < EPL; ++t) {
            const int k = lane + 32 * t;
            rv[t] = fmaf(-alpha, tv[t], rv[t]);
            if (k < r) {
                x[base + k] = fmaf(alpha, pv[t], x[base + k]);
                res[base + k] = rv[t];
            }
            rr = fmaf(rv[t], rv[t], rr);
        }
        rr = warp_sum(rr);
        const float beta = rs_old > 0.f ? rr / rs_old : 0.f;
#pragma unroll
        for (int t = 0; t < EPL; ++t) {
            const int k = lane + 32 * t;
            if (k < r)
                p[base + k] = fmaf(beta, pv[t], rv[t]);
        }
        if (lane == 0)
            rs[row] = rr;
    }
}

// Any r: the same steps with the row streamed from memory three times.
__global__ void __launch_bounds__(256) cg_update_generic(int32_t rows, int32_t r, float lambda,
                                                         float *x, float *res, float *p,
                                                         const float *q, float *rs)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
         row += warps) {
        const size_t base = (size_t)row * r;
        float pq = 0.f;
        for (int k = lane; k < r; k += 32)
            pq = fmaf(p[base + k], fmaf(lambda, p[base + k], q[base + k]), pq);
        pq = warp_sum(pq);
        const float rs_old = rs[row];
        const float alpha = pq > 0.f ? rs_old / pq : 0.f;
        float rr = 0.f;
        for (int k = lane; k < r; k += 32) {
            const float pv = p[base + k];
            const float rv = fmaf(-alpha, fmaf(lambda, pv, q[base + k]), res[base + k]);
            x[base + k] = fmaf(alpha, pv, x[base + k]);
            res[base + k] = rv;
            rr = fmaf(rv, rv, rr);
        }
        rr = warp_sum(rr);
        const float beta = rs_old > 0.f ? rr / rs_old : 0.f;
        for (int k = lane; k < r; k += 32)
            p[base + k] = fmaf(beta, p[base + k], res[base + k]);
        if (lane == 0)
            rs[row] = rr;
    }
}

__global__ void __launch_bounds__(256) cg_init_generic(int32_t rows, int32_t r, float lambda,
                                                       const float *b, const float *mx,
                                                       const float *x, float *res, float *p,
                                                       float *rs)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
         row += warps) {
        const size_t base = (size_t)row * r;
        float acc = 0.f;
        for (int k = lane; k < r; k += 32) {
            const float v = b[base + k] - mx[base + k] - lambda * x[base + k];
            res[base + k] = v;
            p[base + k] = v;
            acc = fmaf(v, v, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0)
            rs[row] = acc;
    }
}

// The same step with float4 vectors: LPR = min(32, r / 4) lanes per row,
// 32 / LPR rows per warp, V = r / (4 LPR) vectors per lane (r a power of two
// from 32 to 256, vectors 16-byte aligned).  Row sums are fixed-order xor
// reductions over the row's lanes.
template <int LPR, int V>
__global__ void __launch_bounds__(256) cg_update_vec(int32_t rows, int32_t r, float lambda,
                                                     float *x, float *res, float *p,
                                                     const float *q, float *rs)
{
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPR - 1);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *r4 = reinterpret_cast<float4 *>(res);
    float4 *p4 = reinterpret_cast<float4 *>(p);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    // warp-uniform loop: every lane takes part in the reductions
    for (int64_t first = warp * RPW; first < rows; first += warps * RPW) {
        const int64_t row = first + lane / LPR;
        const bool ok = row < rows;
        const size_t base = (size_t)row * (r / 4);
        float4 pv[V], tv[V], rv[V];
        float pq = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pv[v] = make_float4(0.f, 0.f, 0.f, 0.f); tv[v] = pv[v]; rv[v] = pv[v];
            if (ok) {
                const size_t i = base + v * LPR + sub;
                pv[v] = p4[i];
                const float4 qv = q4[i];
                tv[v] = make_float4(fmaf(lambda, pv[v].x, qv.x), fmaf(lambda, pv[v].y, qv.y),
                                    fmaf(lambda, pv[v].z, qv.z), fmaf(lambda, pv[v].w, qv.w));
                rv[v] = r4[i];
            }
            pq = fmaf(pv[v].x, tv[v].x, pq); pq = fmaf(pv[v].y, tv[v].y, pq);
            pq = fmaf(pv[v].z, tv[v].z, pq); pq = fmaf(pv[v].w, tv[v].w, pq);
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1)
            pq += __shfl_xor_sync(0xffffffffu, pq, off);
        const float rs_old = ok ? rs[row] : 0.f;
        const float alpha = pq > 0.f ? rs_old / pq : 0.f;
        float rr = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            rv[v].x = fmaf(-alpha, tv[v].x, rv[v].x); rv[v].y = fmaf(-alpha, tv[v].y, rv[v].y);
            rv[v].z = fmaf(-alpha, tv[v].z, rv[v].z); rv[v].w = fmaf(-alpha, tv[v].w, rv[v].w);
            if (ok) {
                const size_t i = base + v * LPR + sub;
                float4 xv = x4[i];
                xv.x = fmaf(alpha, pv[v].x, xv.x); xv.y = fmaf(alpha, pv[v].y, xv.y);
                xv.z = fmaf(alpha, pv[v].z, xv.z); xv.w = fmaf(alpha, pv[v].w, xv.w);
                x4[i] = xv;
                r4[i] = rv[v];
            }
            rr = fmaf(rv[v].x, rv[v].x, rr); rr = fmaf(rv[v].y, rv[v].y, rr);
            rr = fmaf(rv[v].z, rv[v].z, rr); rr = fmaf(rv[v].w, rv[v].w, rr);
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1)
            rr += __shfl_xor_sync(0xffffffffu, rr, off);
        const float beta = rs_old > 0.f ? rr / rs_old : 0.f;
        if (ok) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                p4[base + v * LPR + sub] =
                    make_float4(fmaf(beta, pv[v].x, rv[v].x), fmaf(beta, pv[v].y, rv[v].y),
                                fmaf(beta, pv[v].z, rv[v].z), fmaf(beta, pv[v].w, rv[v].w));
            if (sub == 0)
                rs[row] = rr;
        }
    }
}

static unsigned cg_blocks(int32_t rows)
{
    const int64_t b = ((int64_t)rows + 7) / 8;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), (int64_t)sm_count() * 64);
}

}  // namespace fmm

using namespace fmm;

namespace {

int cg_args(int32_t rows, int32_t r, const void *a, const void *b, const void *c, const void *d,
            const void *e)
{
    if (rows < 0 || r < 1) {
        set_error_msg("cg: rows must be >= 0 and r >= 1");
        return FMM_EINVAL;
    }
    if (rows > 0 && (!a || !b || !c || !d || !e)) {
        set_error_msg("cg: NULL vector");
        return FMM_EINVAL;
    }
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_cg_init(int32_t rows, int32_t r, float lambda, const float *b, const float *mx,
                const float *x, float *res, float *p, float *rs, fmm_stream stream)
{
    int rc = cg_args(rows, r, b, mx, x, res, p);
    if (rc)
        return rc;
    if (rows > 0 && !rs) {
        set_error_msg("cg: NULL rs");
        return FMM_EINVAL;
    }
    if (rows == 0)
        return FMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = cg_blocks(rows);
    if (r <= 32) cg_init_kernel<1><<<g, 256, 0, st>>>(rows, r, lambda, b, mx, x, res, p, rs);
    else if (r <= 64) cg_init_kernel<2><<<g, 256, 0, st>>>(rows, r, lambda, b, mx, x, res, p, rs);
    else if (r <= 128) cg_init_kernel<4><<<g, 256, 0, st>>>(rows, r, lambda, b, mx, x, res, p, rs);
    else if (r <= 256) cg_init_kernel<8><<<g, 256, 0, st>>>(rows, r, lambda, b, mx, x, res, p, rs);
    else cg_init_generic<<<g, 256, 0, st>>>(rows, r, lambda, b, mx, x, res, p, rs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("fmm_cg_init", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

int fmm_cg_update(int32_t rows, int32_t r, float lambda, float *x, float *res, float *p,
                  const float *q, float *rs, fmm_stream stream)
{
    int rc = cg_args(rows, r, x, res, p, q, rs);
    if (rc)
        return rc;
    if (rows == 0)
        return FMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = cg_blocks(rows);
    const bool a16 = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(res) |
                       reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15u) == 0;
    if (a16 && (r == 32 || r == 64 || r == 128 || r == 256)) {
        // rows per warp 32 / LPR: fewer blocks for the same rows
        const int lpr = r / 4 < 32 ? r / 4 : 32;
        const unsigned gv = cg_blocks((int32_t)(((int64_t)rows * lpr + 31) / 32));
        if (r == 32) cg_update_vec<8, 1><<<gv, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
        else if (r == 64) cg_update_vec<16, 1><<<gv, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
        else if (r == 128) cg_update_vec<32, 1><<<gv, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
        else cg_update_vec<32, 2><<<gv, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    } else if (r <= 32) cg_update_kernel<1><<<g, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    else if (r <= 64) cg_update_kernel<2><<<g, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    else if (r <= 128) cg_update_kernel<4><<<g, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    else if (r <= 256) cg_update_kernel<8><<<g, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    else cg_update_generic<<<g, 256, 0, st>>>(rows, r, lambda, x, res, p, q, rs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("fmm_cg_update", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

}  // extern "C"
