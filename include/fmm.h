/*
 * fmm.h -- C ABI of libfmm: FusedMM (an SDDMM feeding an SpMM) on one GPU.
 *
 * Operations (Bharadwaj, Buluc, Demmel, "Distributed-Memory Sparse Kernels
 * for Machine Learning", Sec. II):
 *   SDDMM(A, B, S)  = S * (A B^T), computed only at the nonzeros of S  (Eq. 1)
 *   SpMMA(S, B)     = S B          SpMMB(S, A) = S^T A
 *   FusedMMA(S,A,B) = SpMMA(SDDMM(A, B, S), B)
 *                   : out_i = sum_{(i,j) in nnz(S)} s_ij <A_i, B_j> B_j    (Sec. IV-B)
 *   FusedMMB(S,A,B) = SpMMB(SDDMM(A, B, S), A)
 *                   : out_j = sum_{(i,j) in nnz(S)} s_ij <A_i, B_j> A_i
 * FusedMMB is computed from a transposed copy of the pattern, as the paper
 * does by interchanging A and B and using S^T (Sec. IV-B, last paragraph).
 * The fused kernels keep each SDDMM value in registers, so the intermediate
 * sparse matrix never reaches memory (local kernel fusion, Sec. IV-B (2)).
 *
 * Shapes and layout
 *   S      m x n sparse, CSR: row_ptr[m+1] and col_idx[nnz], int32, on the
 *          device.  row_ptr[0] = 0, row_ptr is nondecreasing, row_ptr[m] = nnz,
 *          0 <= col_idx[p] < n.  Duplicate (i, j) entries are allowed and each
 *          one contributes; columns need not be sorted within a row.
 *   vals   nnz float32 values of S in CSR order, on the device; NULL means
 *          every value is 1.  Values are read on every call, so they may
 *          change between calls on one plan; the pattern may not.
 *   A      m x r, B n x r: dense, row-major, contiguous, on the device, of the
 *          plan's dtype (FMM_F32 = float32, FMM_BF16 = bfloat16 bits).
 *   G, Gn  gradient of a scalar loss with respect to the FusedMMA output
 *          (m x r) or FusedMMB output (n x r): float32, row-major.
 *   out, v, dA, dB, ds: float32, row-major, on the device, caller-owned, and
 *          overwritten (never accumulated into).  Every row of an output is
 *          written, empty rows with zeros.
 * Arithmetic is float32 with float32 accumulation; bfloat16 inputs are
 * widened exactly to float32.  Results are deterministic: the same plan and
 * inputs give bitwise identical outputs on every call (no floating-point
 * atomics).  16-byte aligned dense pointers with r in {32, 64, 128, 256}
 * take the vectorised kernels; any other r or alignment takes a slower
 * generic GPU kernel with the same results up to rounding.  No call ever
 * falls back to the CPU.
 *
 * Streams and ownership
 *   Every compute call is asynchronous on the given stream (a cudaStream_t;
 *   NULL is the legacy default stream) and returns once its kernels are
 *   queued.  The caller owns every buffer it passes and must keep the pattern
 *   (row_ptr, col_idx) alive and unchanged for the life of the plan.  A plan
 *   owns its own device workspace (transposed pattern, schedules, partial
 *   rows of split rows), allocated by fmm_plan_create and freed by
 *   fmm_plan_destroy; compute calls allocate nothing.  Calls on one plan
 *   share that workspace and must be ordered (one stream, or synchronised).
 *
 * Errors
 *   Every entry point returns FMM_OK (0) or a negative status; see
 *   fmm_status_string().  Invalid arguments are reported before anything is
 *   queued.  FMM_ECUDA reports a CUDA runtime error seen while queueing.
 */
#ifndef FMM_H
#define FMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (same underlying type); NULL is the legacy default stream. */
typedef struct CUstream_st *fmm_stream;

enum fmm_status {
    FMM_OK = 0,
    FMM_EINVAL = -1,        /* NULL pointer, negative size, malformed CSR   */
    FMM_EUNSUPPORTED = -2,  /* unknown dtype, r < 1, or a missing S^T       */
    FMM_EOVERFLOW = -3,     /* nnz >= 2^31 or a size that overflows         */
    FMM_ECUDA = -4,         /* CUDA runtime error (launch, copy, device)    */
    FMM_ENOMEM = -5,        /* device allocation failed (plan creation)     */
    FMM_ETIMEOUT = -6       /* a kernel gave up a bounded wait (see
                               fmm_plan_status)                             */
};

enum fmm_dtype {
    FMM_F32 = 0,            /* float32 dense inputs                          */
    FMM_BF16 = 1            /* bfloat16 dense inputs, float32 accumulation   */
};

/* fmm_plan_options.flags */
#define FMM_PLAN_NO_TRANSPOSE 1u  /* skip S^T: the _t and _bwd calls are then FMM_EUNSUPPORTED */

/* Sparse pattern S (device pointers; not copied, referenced by the plan). */
typedef struct fmm_csr {
    int32_t m;                /* rows of S                                */
    int32_t n;                /* columns of S                             */
    int64_t nnz;              /* nonzeros, must be < 2^31                 */
    const int32_t *row_ptr;   /* m + 1 entries                            */
    const int32_t *col_idx;   /* nnz entries                              */
} fmm_csr;

/* Plan options; pass NULL to fmm_plan_create for the defaults. */
typedef struct fmm_plan_options {
    uint32_t flags;           /* FMM_PLAN_* bits                          */
    int32_t split_nnz;        /* rows (and columns, for S^T) with more
                                 nonzeros than this are split into chunks of
                                 this many nonzeros whose partial rows are
                                 summed in a fixed order; 0 = default:
                                 nnz / (4 x the teams of lanes that run at
                                 once for the kernel variant), clamped to
                                 [256, 8192]                                  */
    int32_t variant;          /* kernel variant of the vectorised row passes:
                                 0 = chosen by the plan; else V*100 + N*10 + U
                                 with V = vectors per lane (as a multiple of
                                 the minimum for the row width), N = lane
                                 groups sharing one output row, U = nonzeros
                                 per group per batch; one of 112, 114, 118,
                                 122, 124, 212, 214, 221, 222, 224, 441, 442
                                 (a code that does not fit the row width
                                 falls back to 118); or 1000 + D*10 + V
                                 (1041, 1042, 1081, 1082): FusedMM, SDDMM
                                 and SpMM stage the next D - 1 gathered rows
                                 of each row in shared memory (cp.async);
                                 or F*10000 + M*1000 + P*100 + U*10 + V
                                 (22212, 23212, 22412, 32212, 24221, 34221,
                                 23421, 23241): FusedMM, SDDMM and SpMM keep
                                 the gathered rows of the next P - 1 (F = 2)
                                 or P (F = 3) batches of U nonzeros in
                                 flight in registers, with M resident
                                 256-thread blocks per SM asked for; or
                                 40000 + M*1000 + D*10 + V (44042, 43082,
                                 44041, 44081): FusedMM, SDDMM and SpMM copy
                                 each gathered row into a ring of D slots
                                 in shared memory with one bulk copy
                                 (cp.async.bulk, mbarrier completion), M
                                 resident blocks per SM; or 50000 + M*1000
                                 + P*100 + 10 + V (52212, 52412, 54211):
                                 FusedMM, SDDMM and SpMM walk runs of
                                 consecutive rows (at most 256 nonzeros and
                                 64 rows each, cut by the plan) as one
                                 stream of nonzeros with the register ring
                                 of the F = 3 kind running across row
                                 boundaries.  With these kinds the backward
                                 pass over S^T, and the pass over S except
                                 for 32212 and 52212 (which run it with the
                                 register ring of 32212), run the width's
                                 default team layout (112 for bfloat16
                                 rows, 212 for float32 rows of at most 32
                                 vectors).  The register-ring and streaming
                                 kinds need the gathered operand 32-byte
                                 aligned.  A layout a width does not have
                                 falls back to that team layout.
                                 Default: 32212 for bfloat16 rows of r = 64
                                 and 128, 1042 for float32 rows of r = 128,
                                 else that team layout                       */
} fmm_plan_options;

typedef struct fmm_plan fmm_plan;   /* opaque */

typedef struct fmm_plan_info {
    int32_t m, n, r, dtype;
    int64_t nnz;
    int32_t max_row_nnz;      /* longest row of S                          */
    int32_t max_col_nnz;      /* longest column of S (-1 without S^T)      */
    int32_t split_rows;       /* rows of S split into chunks               */
    int32_t split_cols;       /* columns of S split into chunks            */
    int32_t row_chunks;       /* chunks over the split rows                */
    int32_t col_chunks;       /* chunks over the split columns             */
    int32_t split_nnz;        /* chunk size in nonzeros                    */
    int32_t variant;          /* kernel variant code of passes over S      */
    int32_t variant_t;        /* kernel variant code of passes over S^T    */
    int64_t workspace_bytes;  /* device bytes owned by the plan            */
} fmm_plan_info;

/*
 * Checks a CSR pattern on the device (row_ptr[0] = 0, nondecreasing,
 * row_ptr[m] = nnz, 0 <= col_idx < n).  Synchronises the stream.
 * *first_bad (may be NULL) receives -1 if the pattern is valid, else the
 * smallest offending index: a row_ptr position p as -(p + 2), or a col_idx
 * position p as p.  Returns FMM_OK or FMM_EINVAL (malformed) or an error.
 */
int fmm_csr_validate(const fmm_csr *S, fmm_stream stream, int64_t *first_bad);

/*
 * One-time preprocessing of a pattern, amortised over repeated calls with
 * the same pattern and possibly different values (Sec. I; Sec. III-A on
 * preprocessing amortised by repeated kernel calls).  Validates S (as
 * fmm_csr_validate), builds S^T as CSR with a permutation back to the CSR
 * slots of S (the "two copies, one transposed" of Sec. IV-B), orders rows and
 * columns by length and splits the longest ones into chunks.  r >= 1 is the
 * dense width and dtype an fmm_dtype.  Synchronises the stream; allocates
 * device memory.  *plan receives the plan (NULL on error).
 */
int fmm_plan_create(const fmm_csr *S, int32_t r, int32_t dtype,
                    const fmm_plan_options *options, fmm_stream stream,
                    fmm_plan **plan);

/*
 * Registers values that will not change: copies them once into the order of
 * S^T (a permutation pass, queued on the stream; allocates nnz floats on the
 * first call).  Later calls that pass this same vals pointer skip the
 * per-call permutation of their passes over S^T (fmm_fusedmm_t, fmm_spmm_t
 * with v = vals, the backward passes over S^T) and read the stored copy, so
 * the contents must not change while registered: call again after changing
 * them (or with vals = NULL to forget them).  Values passed through any
 * other pointer are permuted per call as usual.
 */
int fmm_plan_set_values(fmm_plan *plan, const float *vals, fmm_stream stream);

/* Frees a plan and its workspace (synchronises the device first).  NULL is a
 * no-op. */
int fmm_plan_destroy(fmm_plan *plan);

/*
 * Reports and clears the plan's device error word.  Synchronises the stream.
 * Returns FMM_OK, or FMM_ETIMEOUT if a pass of the plan queued before this
 * call gave up waiting for a gathered row to arrive in shared memory (the
 * bulk-staged kernel variants bound every wait; after giving up, the rest
 * of that pass's rows on the affected warp are treated as zeros, so its
 * outputs are wrong).  Status of earlier calls only: compute calls return
 * before their kernels run.
 */
int fmm_plan_status(fmm_plan *plan, fmm_stream stream);

/* Copies the plan's sizes and schedule summary into *info. */
int fmm_plan_get_info(const fmm_plan *plan, fmm_plan_info *info);

/*
 * SDDMM, Sec. II Eq. (1):  v[p] = s_ij * <A_i, B_j>  for the p-th nonzero
 * (i, j) of S in CSR order.  v_out: nnz float32.
 */
int fmm_sddmm(const fmm_plan *plan, const float *vals, const void *A,
              const void *B, float *v_out, fmm_stream stream);

/*
 * SpMMA, Sec. II:  out_i = sum_p v[p] * B_j.  v: nnz float32 in CSR order of
 * S (e.g. the output of fmm_sddmm).  out_m: m x r float32.
 */
int fmm_spmm(const fmm_plan *plan, const float *v, const void *B,
             float *out_m, fmm_stream stream);

/*
 * SpMMB, Sec. II:  out_j = sum_p v[p] * A_i  (S^T A), gathered through S^T.
 * v: nnz float32 in CSR order of S.  out_n: n x r float32.
 */
int fmm_spmm_t(const fmm_plan *plan, const float *v, const void *A,
               float *out_n, fmm_stream stream);

/*
 * FusedMMA, Sec. II and Sec. IV-B:  out_i = sum_j s_ij <A_i, B_j> B_j, one
 * fused kernel (the SDDMM value of a nonzero stays in registers).
 * out_m: m x r float32.
 */
int fmm_fusedmm(const fmm_plan *plan, const float *vals, const void *A,
                const void *B, float *out_m, fmm_stream stream);

/*
 * FusedMMB, Sec. II:  out_j = sum_i s_ij <A_i, B_j> A_i, computed as
 * FusedMMA over S^T with A and B interchanged (Sec. IV-B).  out_n: n x r.
 */
int fmm_fusedmm_t(const fmm_plan *plan, const float *vals, const void *A,
                  const void *B, float *out_n, fmm_stream stream);

/*
 * Adjoint of FusedMMA (not in the paper): gradients of L = <G, FusedMMA>
 * with d = <A_i, B_j>, w = <G_i, B_j> recomputed per nonzero:
 *   ds[p] = d * w,  dA_i = sum_p s_ij w B_j,  dB_j = sum_p s_ij (d G_i + w A_i).
 * G: m x r float32.  dA (m x r), dB (n x r), ds (nnz, CSR order): float32;
 * any of them may be NULL to skip it.  The SDDMM values are never stored.
 */
int fmm_fusedmm_bwd(const fmm_plan *plan, const float *vals, const void *A,
                    const void *B, const float *G, float *dA, float *dB,
                    float *ds, fmm_stream stream);

/*
 * Adjoint of FusedMMB: gradients of L = <Gn, FusedMMB> with
 * d = <A_i, B_j>, w = <Gn_j, A_i>:
 *   ds[p] = d * w,  dB_j = sum_p s_ij w A_i,  dA_i = sum_p s_ij (d Gn_j + w B_j).
 * Gn: n x r float32.  dA, dB, ds as for fmm_fusedmm_bwd.
 */
int fmm_fusedmm_t_bwd(const fmm_plan *plan, const float *vals, const void *A,
                      const void *B, const float *Gn, float *dA, float *dB,
                      float *ds, fmm_stream stream);

/*
 * Accumulating forms, the "+=" of the distributed algorithms (Algorithm 1:
 * each phase adds the contribution of one column block of S to the rows it
 * owns): out_m += FusedMMA, out_n += FusedMMB, dA += and dB += the adjoint
 * of FusedMMA (ds, per nonzero, is overwritten).  The output buffers must
 * hold valid float32 values; otherwise as the plain calls.
 */
int fmm_fusedmm_acc(const fmm_plan *plan, const float *vals, const void *A, const void *B,
                    float *out_m, fmm_stream stream);
int fmm_fusedmm_t_acc(const fmm_plan *plan, const float *vals, const void *A, const void *B,
                      float *out_n, fmm_stream stream);
int fmm_fusedmm_bwd_acc(const fmm_plan *plan, const float *vals, const void *A, const void *B,
                        const float *G, float *dA, float *dB, float *ds, fmm_stream stream);
/* v_out += SDDMM (the partial dot products of one column slice of A and B,
 * summed over the slices by the 1.5D sparse-shifting algorithm, Sec. V);
 * out_m += SpMMA;  out_n += SpMMB. */
int fmm_sddmm_acc(const fmm_plan *plan, const float *vals, const void *A, const void *B,
                  float *v_out, fmm_stream stream);
int fmm_spmm_acc(const fmm_plan *plan, const float *v, const void *B, float *out_m,
                 fmm_stream stream);
int fmm_spmm_t_acc(const fmm_plan *plan, const float *v, const void *A, float *out_n,
                   fmm_stream stream);

/*
 * Kernel variant of a plan's row passes (the codes of
 * fmm_plan_options.variant; 0 leaves a side unchanged).  variant applies to
 * passes over S, variant_t to passes over S^T.  Used by the autotuner; calls
 * already queued are not affected.
 */
int fmm_plan_set_variant(fmm_plan *plan, int32_t variant, int32_t variant_t);

/*
 * Batched FusedMM: many matrices of uneven sizes in one persistent launch
 * per phase (not in the paper; a training-system batching pattern).
 *
 * Each item names a plan and its operands (device pointers, as for
 * fmm_fusedmm and fmm_fusedmm_bwd): vals (NULL = all ones), A (m x r),
 * B (n x r), out (m x r) receive FusedMMA; G (m x r), dA, dB, ds receive its
 * adjoint.  All plans must share one dtype and the current device, have r in
 * {32, 64, 128, 256}, and have no split rows or columns (create them with a
 * split_nnz at least the longest row and column); dense pointers must be
 * 16-byte aligned.  Items without G, or without any gradient output, make a
 * forward-only batch.  The batch stores the pointers: they must stay valid
 * and the buffers at those addresses are read and written by every launch.
 *
 * fmm_batch_forward queues a memset of the batch's work counter and one
 * persistent kernel in which warps pop work units (consecutive rows of one
 * matrix, longest rows of all matrices first) until none are left;
 * fmm_batch_backward does the same for the adjoint passes (over S: dA, ds;
 * over S^T: dB).  Both can be captured in a CUDA graph.  Each item runs the
 * kernel variant its plan selects (fmm_plan_set_variant), if the batch
 * kernels have it for that width and role (codes 112, 114, 122, 212, 214,
 * 221, with at most 32 floats live per lane in the forward phase and 48 in
 * the backward phase), else the width's default with
 * fewer nonzeros per batch.  Results equal the per-item calls with the same variants
 * bit for bit.  Calls on one batch must be ordered (one stream).
 */
typedef struct fmm_batch fmm_batch;   /* opaque */

typedef struct fmm_batch_item {
    const fmm_plan *plan;
    const float *vals;
    const void *A;
    const void *B;
    float *out;
    const float *G;
    float *dA;
    float *dB;
    float *ds;
} fmm_batch_item;

int fmm_batch_create(const fmm_batch_item *items, int32_t count, fmm_stream stream,
                     fmm_batch **batch);
int fmm_batch_forward(const fmm_batch *batch, fmm_stream stream);
int fmm_batch_backward(const fmm_batch *batch, fmm_stream stream);
/* Frees a batch (synchronises the device first).  NULL is a no-op. */
int fmm_batch_destroy(fmm_batch *batch);

/*
 * Row-wise conjugate gradients for ALS (Sec. VI-E).  ALS updates every row x_i
 * of one factor by solving M_i x_i = b_i, M_i x = sum_j <x, Y_j> Y_j +
 * lambda x, b_i = sum_j c_ij Y_j over the nonzeros of the row (the other
 * factor Y fixed).  CG runs on all rows at once: the product M p of every row
 * without the lambda term is one FusedMM over the 0/1 pattern (fmm_fusedmm
 * with vals = NULL for the A side, fmm_fusedmm_t for the B side), b is one
 * SpMM of the observed values (fmm_spmm / fmm_spmm_t), and these two calls do
 * the per-row vector work of a CG step in one kernel.
 *
 * All vectors are float32, rows x r, row-major, on the device; rs holds one
 * float per row.
 * fmm_cg_init:   res = b - mx - lambda x;  p = res;  rs = <res, res>
 *                (mx = the FusedMM of x, without the lambda term).
 * fmm_cg_update: with q = the FusedMM of p (without lambda), t = q + lambda p:
 *                alpha = rs / <p, t> (0 if <p, t> <= 0);  x += alpha p;
 *                res -= alpha t;  rs' = <res, res>;  beta = rs' / rs (0 if
 *                rs = 0);  p = res + beta p;  rs = rs'.
 * Row reductions are fixed-order warp sums: results are deterministic.
 */
int fmm_cg_init(int32_t rows, int32_t r, float lambda, const float *b, const float *mx,
                const float *x, float *res, float *p, float *rs, fmm_stream stream);
int fmm_cg_update(int32_t rows, int32_t r, float lambda, float *x, float *res, float *p,
                  const float *q, float *rs, fmm_stream stream);

/*
 * Graph-attention layer, forward (Sec. VI-E, the GAT workload): the attention
 * variant of SDDMM feeding a softmax-normalised SpMM.  For every head h
 * (heads must divide the plan's r; head h owns columns [h*rh, (h+1)*rh) with
 * rh = r / heads) and nonzero (i, j):
 *   e_ij = LeakyReLU(s_ij (f_i + g_j))       (LeakyReLU(x) = x > 0 ? x : slope x)
 *   out_i = sum_j softmax_j(e_i.)_j  H_j      (softmax over the nonzeros of row i)
 * f (m x heads) and g (n x heads) are the per-node projections a_l^T H_i and
 * a_r^T H_j that make up the paper's a^T (H_i || H_j); H (n x r) of the
 * plan's dtype; out (m x r) float32; vals NULL = all ones.  Rows without
 * nonzeros give zeros.  One gather pass per row with an online softmax.
 */
int fmm_gat_forward(const fmm_plan *plan, int32_t heads, const float *vals, const float *f,
                    const float *g, const void *H, float slope, float *out, fmm_stream stream);

/* out[i, h] = sum_k X[i, h*rh + k] w[h*rh + k]  (rows x heads, float32): the
 * per-node projections f and g of fmm_gat_forward. */
int fmm_gat_project(int32_t rows, int32_t heads, int32_t rh, const float *X, const float *w,
                    float *out, fmm_stream stream);

/*
 * FusedMMA (same result as fmm_fusedmm) for callers that cannot allocate
 * device memory: no plan, no cudaMalloc, no allocating library call.  The
 * paper has no counterpart; this is an interface for memory-constrained
 * callers (a caller inside a pool or arena that owns all device memory, or a
 * runtime that forbids allocation on its hot path).
 *
 * S (a valid pattern, see fmm_csr_validate; a malformed one gives
 * unspecified results but no out-of-bounds access), r >= 1, dtype, vals
 * (NULL = all ones), A (m x r), B (n x r) and out_m (m x r, float32) are as
 * for fmm_plan_create and fmm_fusedmm.  The only scratch is a fixed
 * file-scope device array of 34,603,264 bytes per device (held by every
 * device that loads the library's module until exit): rows longer than
 * ch = max(512, ceil(2 nnz / min(65536, 8388608 / r))) nonzeros are split
 * into chunks whose partial rows live there.  r > 65536 returns
 * FMM_EOVERFLOW.  The array is shared by all calls: calls that overlap on the
 * GPU race and give wrong results, so order them on one stream.  Every
 * call looks the array's address up (cudaGetSymbolAddress, which allocates
 * nothing) on the current device, so the call still finds it after
 * cudaDeviceReset; the first call on a device may load the library's module
 * there, so make that first call before any stream capture.
 * Asynchronous on the stream; deterministic.
 */
int fmm_fusedmm_noalloc(const fmm_csr *S, int32_t r, int32_t dtype, const float *vals,
                        const void *A, const void *B, float *out_m, fmm_stream stream);

/*
 * Gather-rate probe (a measurement aid; the paper has no counterpart): for
 * k < count, fetches row idx[k] (row_bytes bytes, 16-byte vectors, the
 * read-only path the row passes use) of `table` (rows x row_bytes, 16-byte
 * aligned, device) and does nothing else with it, so its time is the
 * ceiling for the gather part of a row pass walking the same index list.
 * row_bytes is 64, 128, 256 or 512; idx (count int32, device) is clamped
 * into [0, rows).  sink (one uint32, device) may be written.  Asynchronous
 * on the stream.
 */
int fmm_probe_gather(const void *table, int64_t rows, int32_t row_bytes, const int32_t *idx,
                     int64_t count, uint32_t *sink, fmm_stream stream);

/* Static description of a status code (never NULL). */
const char *fmm_status_string(int status);

/* Message of the last error seen by this thread's calls ("" if none). */
const char *fmm_last_error(void);

/* ABI version of this header: (major << 16) | minor. */
int32_t fmm_version(void);

#define FMM_VERSION ((1 << 16) | 0)

#ifdef __cplusplus
}
#endif

#endif /* FMM_H */
