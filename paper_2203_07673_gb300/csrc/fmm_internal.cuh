// Internal declarations shared by the libfmm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fmm.h"

namespace fmm {

// Kernel variant of the vectorised row passes: vectors per lane (as a
// multiple of the row shape's minimum), groups per team, nonzeros per group
// per batch.
struct KernelVariant {
    int vpl_mult = 1, ng = 1, u = 8;
    int stages = 0;   // > 0: the staged pass (fmm_staged.cuh) with this ring depth
    int ring = 0;     // > 0: the pipelined pass (fmm_pipe.cuh), this many batches in
                      // the register ring (forward roles; u nonzeros per batch)
    int mb = 0;       // pipelined pass: resident 256-thread blocks per SM asked for
    int refill = 0;   // pipelined pass: 1 = refill a slot as soon as it is read
    int depth = 0;    // > 0: the bulk-staged pass (fmm_bulk.cuh), this many row
                      // slots in shared memory per team (forward roles)
    int stream = 0;   // 1: the streaming pass (fmm_stream.cuh): a team walks a run
                      // of consecutive rows as one stream of nonzeros, with the
                      // register ring of the pipelined pass (ring, mb; refill)
};

// One side of a plan: the CSR that a row pass walks (S itself, or S^T with a
// permutation back to the CSR slots of S) plus its schedule.
struct Side {
    int32_t rows = 0;                 // rows of this CSR (m for S, n for S^T)
    const int32_t *row_ptr = nullptr; // rows + 1
    const int32_t *col_idx = nullptr; // nnz
    const int32_t *perm = nullptr;    // nnz; NULL on the S side (identity)
    int32_t *order = nullptr;         // rows: split rows first, then the rest in
                                      // length buckets (length_key), index order
                                      // within a bucket
    int32_t n_split = 0;              // rows split into chunks
    int32_t n_light = 0;              // rows - n_split
    int4 *chunks = nullptr;           // {row, begin, end, unused} per chunk
    int32_t n_chunks = 0;
    int4 *split = nullptr;            // {row, first chunk, chunk count, unused}
    int2 *runs = nullptr;             // {first row, end row}: runs of consecutive
                                      // light rows for the streaming pass
    int32_t n_runs = 0;
    float *partials = nullptr;        // 3 x n_chunks x r floats: partial rows (and
                                      // the attention pass's softmax states)
    int32_t max_nnz = 0;              // longest row
    KernelVariant variant;            // kernel variant of passes over this side
    std::vector<int32_t> bucket_start;  // host: first position in `order` of
                                        // each length key (257 entries)
    const int32_t *light_order() const { return order ? order + n_split : nullptr; }
};

// Length key of a row for the plan's row order (ascending key = longer rows
// first): 0 for split rows, 255 for empty rows, else 254 - q(d) with q(d) =
// d - 1 for d < 4 and 3 + 4 (k - 2) + the two bits after the leading one for
// 2^k <= d < 2^(k+1): four buckets per power of two, so rows of one bucket
// differ in length by less than a quarter.
__host__ __device__ inline uint32_t length_key(int32_t d, int32_t split_nnz)
{
    if (d > split_nnz) return 0u;
    if (d <= 0) return 255u;
    if (d < 4) return 254u - (uint32_t)(d - 1);
    int k = 31;
    while (!((uint32_t)d >> k)) --k;
    const uint32_t sub = ((uint32_t)d >> (k - 2)) & 3u;
    return 254u - (3u + 4u * (uint32_t)(k - 2) + sub);
}

// Shortest row length of a length key in [136, 254].
inline int32_t length_key_min(uint32_t key)
{
    const uint32_t q = 254u - key;
    if (q < 3) return (int32_t)q + 1;
    const int k = (int)((q - 3) / 4) + 2;
    const int sub = (int)((q - 3) % 4);
    return (1 << k) + sub * (1 << (k - 2));
}

// Kernel roles.  "local" rows belong to the row being produced; "gathered"
// rows are fetched per nonzero through col_idx.
enum Mode : int {
    M_FUSED = 0,    // acc += s * <L_i, Y_j> * Y_j
    M_SDDMM = 1,    // nzout[p] = s * <L_i, Y_j>
    M_SPMM = 2,     // acc += s * Y_j            (s = the SDDMM values)
    M_BWD_ROW = 3,  // d = <L_i,Y_j>, w = <H_i,Y_j>: nzout[p] = d w, acc += s w Y_j
    M_BWD_COL = 4   // d = <Y_i,L_j>, w = <H_i,L_j>: acc += s (d H_i + w Y_i)
};

struct PassArgs {
    // pattern walked
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *perm;       // maps a slot of this CSR to the CSR slot of S
    const int32_t *order;      // light rows in processing order
    int32_t n_light;
    const int4 *chunks;
    int32_t n_chunks;
    float *partials;
    const int2 *runs = nullptr;  // runs of consecutive light rows (streaming pass)
    int32_t n_runs = 0;
    // operands
    const float *s;            // per-nonzero scalars (NULL = 1): in S order, or in
                               // this CSR's order when s_direct is set
    int32_t s_direct;
    const void *L;             // local rows (dtype of the plan)
    const void *Y;             // gathered rows (dtype of the plan)
    const float *H;            // float32 gradient rows (local or gathered)
    float *out;                // rows x r (NULL: not stored)
    float *nzout;              // per-nonzero output in S order (NULL: none)
    int32_t r;
    int32_t *err = nullptr;    // device word set to 1 by a pass that gave up a
                               // bounded wait (NULL: not reported)
    int32_t accumulate = 0;    // 1: out += the pass's rows (else out =)
};

// Launches one row pass (main kernel; the combine kernel for split rows is
// separate).  dtype: FMM_F32 / FMM_BF16.
cudaError_t launch_pass(int mode, int dtype, const KernelVariant &v, const PassArgs &a,
                        cudaStream_t st);
cudaError_t launch_pass_f32(int mode, int vpl_mult, int ng, int u, bool vec, const PassArgs &a,
                            cudaStream_t st);
cudaError_t launch_pass_bf16(int mode, int vpl_mult, int ng, int u, bool vec, const PassArgs &a,
                             cudaStream_t st);
// Staged forward-role passes (fmm_staged.cuh): FusedMM, SDDMM and SpMM with a
// cp.async ring of `stages` gathered rows per team; vector path only.
cudaError_t launch_staged_f32(int mode, int vpl_mult, int stages, const PassArgs &a,
                              cudaStream_t st);
cudaError_t launch_staged_bf16(int mode, int vpl_mult, int stages, const PassArgs &a,
                               cudaStream_t st);
// Pipelined forward-role passes (fmm_pipe.cuh): FusedMM, SDDMM and SpMM with
// a register ring of `ring` batches of u gathered rows per team; vector path.
// Bulk-staged forward-role passes (fmm_bulk.cuh): rows copied into a
// shared-memory ring of `depth` slots per team by cp.async.bulk.
cudaError_t launch_bulk_f32(int mode, int vpl_mult, int depth, int mb, const PassArgs &a,
                            cudaStream_t st);
cudaError_t launch_bulk_bf16(int mode, int vpl_mult, int depth, int mb, const PassArgs &a,
                             cudaStream_t st);
cudaError_t launch_pipe_f32(int mode, int vpl_mult, int u, int ring, int mb, int refill,
                            const PassArgs &a, cudaStream_t st);
cudaError_t launch_stream_f32(int mode, int vpl_mult, int ring, int mb, const PassArgs &a,
                              cudaStream_t st);
cudaError_t launch_stream_bf16(int mode, int vpl_mult, int ring, int mb, const PassArgs &a,
                               cudaStream_t st);
// Runs of the streaming pass: consecutive light rows with at most this many
// nonzeros together (a longer light row is a run of its own) and at most
// kRunRows rows.
constexpr int32_t kRunNnz = 256;
constexpr int32_t kRunRows = 64;
cudaError_t launch_pipe_bf16(int mode, int vpl_mult, int u, int ring, int mb, int refill,
                             const PassArgs &a, cudaStream_t st);
// dst[q] = src[perm[q]] for q < nnz (values of S into the order of S^T).
cudaError_t launch_permute(const float *src, const int32_t *perm, float *dst, int64_t nnz,
                           cudaStream_t st);
// Values of S in the order of S^T for a plan: the windowed two-pass
// permutation where the plan has it, else launch_permute.
cudaError_t launch_values_t(const fmm_plan *p, const float *src, float *dst, cudaStream_t st);
// S^T slots per window of the windowed permutation (32 MB of float32 values:
// a window's staging values stay in L2 while its slots are filled).
constexpr int64_t kPermuteWindow = int64_t(1) << 23;
// Sums the partial rows of every split row, in chunk order, into out (added
// to out's rows when accumulate is set).
cudaError_t launch_combine(const Side &side, float *out, int32_t r, bool accumulate,
                           cudaStream_t st);

bool fast_r(int32_t r);
// Streaming multiprocessors of the current device (queried once per device;
// 1 if the query fails, which keeps grid-stride launches correct).
int sm_count();
bool variant_known(int code);
KernelVariant decode_variant(int code);
int encode_variant(const KernelVariant &v);
// Default kernel variant of a pass over rows of width r (dtype, average
// nonzeros per row).
KernelVariant default_variant(int32_t r, int32_t dtype, double avg_nnz);
// The team kernel's layout for a width (one group per row, 8 elements per
// lane, 2 nonzeros per batch): the default of the batch kernels.
KernelVariant team_default_variant(int32_t r, int32_t dtype);
// Default split size of long rows for a pattern of nnz nonzeros and rows of
// width r run with variant v.
int32_t default_split_nnz(int64_t nnz, int32_t r, int32_t dtype, const KernelVariant &v);

// Plan construction and error reporting (fmm_plan.cu).
int check_csr_args(const fmm_csr *S);
int validate_csr(const fmm_csr *S, cudaStream_t st, int64_t *first_bad);
int create_plan(const fmm_csr *S, int32_t r, int32_t dtype, const fmm_plan_options *opt,
                cudaStream_t st, fmm_plan **out);
void destroy_plan(fmm_plan *p);
void set_error(const char *what, cudaError_t e);
void set_error_msg(const char *what);
const char *last_error();

}  // namespace fmm

struct fmm_plan {
    int32_t m = 0, n = 0, r = 0, dtype = 0;
    int64_t nnz = 0;
    uint32_t flags = 0;
    int32_t split_nnz = 512;
    int32_t variant = 0;              // requested variant code (0 = default)
    bool has_t = false;
    fmm::Side rows;   // S
    fmm::Side cols;   // S^T
    int32_t *row_ptr_t = nullptr;
    int32_t *col_idx_t = nullptr;
    int32_t *perm_t = nullptr;
    float *vals_t = nullptr;          // per-call values permuted into S^T order
    const float *static_src = nullptr;  // values registered by fmm_plan_set_values
    float *vals_static = nullptr;       // ... and their copy in S^T order
    int64_t workspace_bytes = 0;
    int device = 0;
    int32_t *err = nullptr;           // device word: a pass gave up a bounded wait
    // windowed value permutation (plans with more than 2 windows of
    // nonzeros): S-order slot p -> its place in the window staging array,
    // S^T slot q -> where its value waits there, and the staging array
    int32_t *win_pos1 = nullptr;
    int32_t *win_pos2 = nullptr;
    float *win_tmp = nullptr;
};
