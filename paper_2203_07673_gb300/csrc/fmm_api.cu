// C-ABI entry points of libfmm (declared in include/fmm.h).
#include <atomic>
#include <cstdint>
#include <cstdio>

#include "fmm_internal.cuh"

namespace fmm {

bool fast_r(int32_t r) { return r == 32 || r == 64 || r == 128 || r == 256; }

int sm_count()
{
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    if (dev >= 0 && dev < 64) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0)
            return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        return 1;
    if (dev >= 0 && dev < 64)
        cached[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
static bool aligned32(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 31u) == 0; }

// Variant codes: vectors-per-lane multiple * 100 + groups per team * 10 +
// nonzeros per group per batch (the combinations instantiated in
// fmm_rows.cuh; a combination that does not fit a row shape falls back to
// the shape's default); 1000 + ring depth * 10 + vectors-per-lane multiple
// for the staged pass (fmm_staged.cuh); (2 + refill) * 10000 + resident
// blocks per SM * 1000 + register-ring batches * 100 + nonzeros per batch *
// 10 + vectors-per-lane multiple for the pipelined pass (fmm_pipe.cuh);
// 40000 + resident blocks per SM * 1000 + ring slots * 10 + vectors-per-lane
// multiple for the bulk-staged pass (fmm_bulk.cuh); 50000 + resident blocks
// per SM * 1000 + register-ring batches * 100 + 10 + vectors-per-lane
// multiple for the streaming pass (fmm_stream.cuh, one nonzero per batch,
// refill order).  The backward roles of staged and bulk-staged codes run
// the team kernel in the width's default layout (team_default_variant);
// pipelined and streaming codes run the adjoint pass over S by the
// pipelined pass of the same ring (where instantiated) and the pass over
// S^T by the team kernel.
static const int kVariantCodes[] = {114, 118, 222, 224, 441, 442, 214, 124, 112, 122, 212, 221,
                                    1041, 1042, 1081, 1082,
                                    22212, 23212, 22412, 32212, 24221, 34221, 23421, 23241,
                                    44042, 43082, 44041, 44081, 52212, 52412, 54211};

bool variant_known(int code)
{
    for (int c : kVariantCodes)
        if (c == code) return true;
    return false;
}

KernelVariant decode_variant(int code)
{
    KernelVariant v;
    if (code >= 50000) {
        v.stream = 1;
        v.refill = 1;
        v.mb = (code / 1000) % 10;
        v.ring = (code / 100) % 10;
        v.u = 1;
        v.vpl_mult = code % 10;
        v.ng = 1;
        return v;
    }
    if (code >= 40000) {
        v.mb = (code / 1000) % 10;
        v.depth = (code / 10) % 100;
        v.vpl_mult = code % 10;
        v.ng = 1;
        v.u = 2;
        return v;
    }
    if (code >= 20000) {
        v.refill = code / 10000 - 2;
        v.mb = (code / 1000) % 10;
        v.ring = (code / 100) % 10;
        v.u = (code / 10) % 10;
        v.vpl_mult = code % 10;
        v.ng = 1;
        return v;
    }
    if (code >= 1000) {
        v.stages = (code / 10) % 100;
        v.vpl_mult = code % 10;
        v.ng = 1;
        v.u = 2;
        return v;
    }
    v.vpl_mult = code / 100;
    v.ng = (code / 10) % 10;
    v.u = code % 10;
    return v;
}

int encode_variant(const KernelVariant &v)
{
    if (v.stream)
        return 50000 + v.mb * 1000 + v.ring * 100 + 10 + v.vpl_mult;
    if (v.depth > 0)
        return 40000 + v.mb * 1000 + v.depth * 10 + v.vpl_mult;
    if (v.ring > 0)
        return (2 + v.refill) * 10000 + v.mb * 1000 + v.ring * 100 + v.u * 10 + v.vpl_mult;
    if (v.stages > 0)
        return 1000 + v.stages * 10 + v.vpl_mult;
    return v.vpl_mult * 100 + v.ng * 10 + v.u;
}

cudaError_t launch_pass(int mode, int dtype, const KernelVariant &v, const PassArgs &a,
                        cudaStream_t st)
{
    const bool vec = fast_r(a.r) && aligned16(a.L) && aligned16(a.Y) && aligned16(a.H) &&
                     aligned16(a.out) && aligned16(a.partials);
    const bool fwd = mode == M_FUSED || mode == M_SDDMM || mode == M_SPMM;
    if (v.stages > 0 && vec && fwd) {
        return dtype == FMM_BF16 ? launch_staged_bf16(mode, v.vpl_mult, v.stages, a, st)
                                 : launch_staged_f32(mode, v.vpl_mult, v.stages, a, st);
    }
    if (v.stream && vec && fwd && aligned32(a.Y)) {
        const cudaError_t e = dtype == FMM_BF16
                                  ? launch_stream_bf16(mode, v.vpl_mult, v.ring, v.mb, a, st)
                                  : launch_stream_f32(mode, v.vpl_mult, v.ring, v.mb, a, st);
        if (e != cudaErrorNotSupported)
            return e;
    }
    if (v.depth > 0 && vec && fwd) {
        const cudaError_t e = dtype == FMM_BF16
                                  ? launch_bulk_bf16(mode, v.vpl_mult, v.depth, v.mb, a, st)
                                  : launch_bulk_f32(mode, v.vpl_mult, v.depth, v.mb, a, st);
        if (e != cudaErrorNotSupported)
            return e;
    }
    // the register-ring pass loads gathered rows 32 bytes at a time; of the
    // adjoint roles it has the pass over S
    if (v.ring > 0 && vec && (fwd || mode == M_BWD_ROW) && aligned32(a.Y)) {
        const cudaError_t e = dtype == FMM_BF16
                                  ? launch_pipe_bf16(mode, v.vpl_mult, v.u, v.ring, v.mb, v.refill, a, st)
                                  : launch_pipe_f32(mode, v.vpl_mult, v.u, v.ring, v.mb, v.refill, a, st);
        if (e != cudaErrorNotSupported)
            return e;
        // a ring layout this width does not have: the team kernel below
    }
    // other backward roles of a staged, pipelined or bulk-staged plan: the
    // team kernel's default layout for the width
    const KernelVariant t =
        (v.stages > 0 || v.ring > 0 || v.depth > 0) ? team_default_variant(a.r, dtype) : v;
    if (dtype == FMM_BF16)
        return launch_pass_bf16(mode, t.vpl_mult, t.ng, t.u, vec, a, st);
    return launch_pass_f32(mode, t.vpl_mult, t.ng, t.u, vec, a, st);
}

}  // namespace fmm

using namespace fmm;

namespace {

int check_plan(const fmm_plan *p)
{
    if (!p) {
        set_error_msg("plan is NULL");
        return FMM_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("cudaGetDevice", e);
        return FMM_ECUDA;
    }
    if (dev != p->device) {
        set_error_msg("current device differs from the plan's device");
        return FMM_EINVAL;
    }
    return FMM_OK;
}

// A dense operand with `rows` rows may be NULL only when it has no rows.
int need(const void *ptr, int64_t rows, const char *name)
{
    if (!ptr && rows > 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "%s is NULL", name);
        set_error_msg(msg);
        return FMM_EINVAL;
    }
    return FMM_OK;
}

int need_t(const fmm_plan *p)
{
    if (!p->has_t) {
        set_error_msg("plan built with FMM_PLAN_NO_TRANSPOSE");
        return FMM_EUNSUPPORTED;
    }
    return FMM_OK;
}

int run_pass(const fmm_plan *p, const Side &side, int mode, const float *s, const void *L,
             const void *Y, const float *H, float *out, float *nzout, cudaStream_t st,
             bool accumulate = false)
{
    PassArgs a;
    a.row_ptr = side.row_ptr;
    a.col_idx = side.col_idx;
    a.perm = side.perm;
    a.order = side.light_order();
    a.n_light = side.n_light;
    a.chunks = side.chunks;
    a.n_chunks = side.n_chunks;
    a.partials = side.partials;
    a.runs = side.runs;
    a.n_runs = side.n_runs;
    a.s = s;
    a.s_direct = 0;
    a.L = L;
    a.Y = Y;
    a.H = H;
    a.out = out;
    a.nzout = nzout;
    a.r = p->r;
    a.err = p->err;
    a.accumulate = accumulate ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (side.perm && s) {
        if (s == p->static_src && p->vals_static) {
            // registered values: their S^T-order copy is already there
            a.s = p->vals_static;
        } else {
            // values of S gathered once into the order of S^T, so the pass
            // streams them instead of fetching one scattered word per nonzero
            e = launch_values_t(p, s, p->vals_t, st);
            a.s = p->vals_t;
        }
        a.s_direct = 1;
    }
    if (e == cudaSuccess)
        e = launch_pass(mode, p->dtype, side.variant, a, st);
    if (e == cudaSuccess && mode != M_SDDMM)
        e = launch_combine(side, out, p->r, accumulate, st);
    if (e != cudaSuccess) {
        set_error("kernel launch", e);
        return FMM_ECUDA;
    }
    return FMM_OK;
}

#define CHECK(x)              \
    do {                      \
        int _rc = (x);        \
        if (_rc) return _rc;  \
    } while (0)

}  // namespace

extern "C" {

int fmm_csr_validate(const fmm_csr *S, fmm_stream stream, int64_t *first_bad)
{
    if (first_bad) *first_bad = -1;
    CHECK(check_csr_args(S));
    return validate_csr(S, (cudaStream_t)stream, first_bad);
}

int fmm_plan_create(const fmm_csr *S, int32_t r, int32_t dtype, const fmm_plan_options *options,
                    fmm_stream stream, fmm_plan **plan)
{
    if (!plan) {
        set_error_msg("plan output pointer is NULL");
        return FMM_EINVAL;
    }
    *plan = nullptr;
    CHECK(check_csr_args(S));
    if (r < 1) {
        set_error_msg("r must be >= 1");
        return FMM_EUNSUPPORTED;
    }
    if (dtype != FMM_F32 && dtype != FMM_BF16) {
        set_error_msg("unknown dtype");
        return FMM_EUNSUPPORTED;
    }
    if ((int64_t)std::max(S->m, S->n) * r >= (int64_t(1) << 40)) {
        set_error_msg("dense operand too large");
        return FMM_EOVERFLOW;
    }
    if (options) {
        if (options->split_nnz < 0 ||
            (options->variant != 0 && !variant_known(options->variant)) ||
            (options->flags & ~FMM_PLAN_NO_TRANSPOSE)) {
            set_error_msg("invalid plan options");
            return FMM_EINVAL;
        }
    }
    CHECK(validate_csr(S, (cudaStream_t)stream, nullptr));
    return create_plan(S, r, dtype, options, (cudaStream_t)stream, plan);
}

int fmm_plan_set_values(fmm_plan *p, const float *vals, fmm_stream stream)
{
    CHECK(check_plan(p));
    p->static_src = nullptr;
    if (!vals || !p->has_t || p->nnz == 0)
        return FMM_OK;
    if (!p->vals_static) {
        cudaError_t e = cudaMalloc(&p->vals_static, sizeof(float) * (size_t)p->nnz);
        if (e != cudaSuccess) {
            p->vals_static = nullptr;
            set_error("allocate registered values", e);
            return e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA;
        }
        p->workspace_bytes += (int64_t)sizeof(float) * p->nnz;
    }
    cudaError_t e = launch_values_t(p, vals, p->vals_static, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("fmm_plan_set_values", e);
        return FMM_ECUDA;
    }
    p->static_src = vals;
    return FMM_OK;
}

int fmm_plan_destroy(fmm_plan *plan)
{
    destroy_plan(plan);
    return FMM_OK;
}

int fmm_plan_get_info(const fmm_plan *p, fmm_plan_info *info)
{
    if (!p || !info) {
        set_error_msg("NULL argument");
        return FMM_EINVAL;
    }
    info->m = p->m;
    info->n = p->n;
    info->r = p->r;
    info->dtype = p->dtype;
    info->nnz = p->nnz;
    info->max_row_nnz = p->rows.max_nnz;
    info->max_col_nnz = p->has_t ? p->cols.max_nnz : -1;
    info->split_rows = p->rows.n_split;
    info->split_cols = p->cols.n_split;
    info->row_chunks = p->rows.n_chunks;
    info->col_chunks = p->cols.n_chunks;
    info->split_nnz = p->split_nnz;
    info->variant = encode_variant(p->rows.variant);
    info->variant_t = p->has_t ? encode_variant(p->cols.variant) : 0;
    info->workspace_bytes = p->workspace_bytes;
    return FMM_OK;
}

static int sddmm_(const fmm_plan *p, const float *vals, const void *A, const void *B,
                  float *v_out, fmm_stream stream, bool acc)
{
    CHECK(check_plan(p));
    CHECK(need(A, p->m, "A"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(v_out, p->nnz, "v_out"));
    return run_pass(p, p->rows, M_SDDMM, vals, A, B, nullptr, nullptr, v_out,
                    (cudaStream_t)stream, acc);
}

static int spmm_(const fmm_plan *p, const float *v, const void *B, float *out_m,
                 fmm_stream stream, bool acc)
{
    CHECK(check_plan(p));
    CHECK(need(v, p->nnz, "v"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(out_m, p->m, "out_m"));
    return run_pass(p, p->rows, M_SPMM, v, nullptr, B, nullptr, out_m, nullptr,
                    (cudaStream_t)stream, acc);
}

static int spmm_t_(const fmm_plan *p, const float *v, const void *A, float *out_n,
                   fmm_stream stream, bool acc)
{
    CHECK(check_plan(p));
    CHECK(need_t(p));
    CHECK(need(v, p->nnz, "v"));
    CHECK(need(A, p->m, "A"));
    CHECK(need(out_n, p->n, "out_n"));
    return run_pass(p, p->cols, M_SPMM, v, nullptr, A, nullptr, out_n, nullptr,
                    (cudaStream_t)stream, acc);
}

int fmm_sddmm(const fmm_plan *p, const float *vals, const void *A, const void *B, float *v_out,
              fmm_stream stream)
{
    return sddmm_(p, vals, A, B, v_out, stream, false);
}

int fmm_spmm(const fmm_plan *p, const float *v, const void *B, float *out_m, fmm_stream stream)
{
    return spmm_(p, v, B, out_m, stream, false);
}

int fmm_spmm_t(const fmm_plan *p, const float *v, const void *A, float *out_n, fmm_stream stream)
{
    return spmm_t_(p, v, A, out_n, stream, false);
}

int fmm_sddmm_acc(const fmm_plan *p, const float *vals, const void *A, const void *B,
                  float *v_out, fmm_stream stream)
{
    return sddmm_(p, vals, A, B, v_out, stream, true);
}

int fmm_spmm_acc(const fmm_plan *p, const float *v, const void *B, float *out_m,
                 fmm_stream stream)
{
    return spmm_(p, v, B, out_m, stream, true);
}

int fmm_spmm_t_acc(const fmm_plan *p, const float *v, const void *A, float *out_n,
                   fmm_stream stream)
{
    return spmm_t_(p, v, A, out_n, stream, true);
}

static int fusedmm_a(const fmm_plan *p, const float *vals, const void *A, const void *B,
                     float *out_m, fmm_stream stream, bool acc)
{
    CHECK(check_plan(p));
    CHECK(need(A, p->m, "A"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(out_m, p->m, "out_m"));
    return run_pass(p, p->rows, M_FUSED, vals, A, B, nullptr, out_m, nullptr,
                    (cudaStream_t)stream, acc);
}

static int fusedmm_b(const fmm_plan *p, const float *vals, const void *A, const void *B,
                     float *out_n, fmm_stream stream, bool acc)
{
    CHECK(check_plan(p));
    CHECK(need_t(p));
    CHECK(need(A, p->m, "A"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(out_n, p->n, "out_n"));
    return run_pass(p, p->cols, M_FUSED, vals, B, A, nullptr, out_n, nullptr,
                    (cudaStream_t)stream, acc);
}

static int fusedmm_a_bwd(const fmm_plan *p, const float *vals, const void *A, const void *B,
                         const float *G, float *dA, float *dB, float *ds, fmm_stream stream,
                         bool acc)
{
    CHECK(check_plan(p));
    CHECK(need(A, p->m, "A"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(G, p->m, "G"));
    if (dB)
        CHECK(need_t(p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dA || ds)
        CHECK(run_pass(p, p->rows, M_BWD_ROW, vals, A, B, G, dA, ds, st, acc));
    if (dB)
        CHECK(run_pass(p, p->cols, M_BWD_COL, vals, B, A, G, dB, nullptr, st, acc));
    return FMM_OK;
}

int fmm_fusedmm(const fmm_plan *p, const float *vals, const void *A, const void *B, float *out_m,
                fmm_stream stream)
{
    return fusedmm_a(p, vals, A, B, out_m, stream, false);
}

int fmm_fusedmm_t(const fmm_plan *p, const float *vals, const void *A, const void *B,
                  float *out_n, fmm_stream stream)
{
    return fusedmm_b(p, vals, A, B, out_n, stream, false);
}

int fmm_fusedmm_bwd(const fmm_plan *p, const float *vals, const void *A, const void *B,
                    const float *G, float *dA, float *dB, float *ds, fmm_stream stream)
{
    return fusedmm_a_bwd(p, vals, A, B, G, dA, dB, ds, stream, false);
}

int fmm_fusedmm_acc(const fmm_plan *p, const float *vals, const void *A, const void *B,
                    float *out_m, fmm_stream stream)
{
    return fusedmm_a(p, vals, A, B, out_m, stream, true);
}

int fmm_fusedmm_t_acc(const fmm_plan *p, const float *vals, const void *A, const void *B,
                      float *out_n, fmm_stream stream)
{
    return fusedmm_b(p, vals, A, B, out_n, stream, true);
}

int fmm_fusedmm_bwd_acc(const fmm_plan *p, const float *vals, const void *A, const void *B,
                        const float *G, float *dA, float *dB, float *ds, fmm_stream stream)
{
    return fusedmm_a_bwd(p, vals, A, B, G, dA, dB, ds, stream, true);
}

int fmm_fusedmm_t_bwd(const fmm_plan *p, const float *vals, const void *A, const void *B,
                      const float *Gn, float *dA, float *dB, float *ds, fmm_stream stream)
{
    CHECK(check_plan(p));
    CHECK(need(A, p->m, "A"));
    CHECK(need(B, p->n, "B"));
    CHECK(need(Gn, p->n, "Gn"));
    if (dB || ds)
        CHECK(need_t(p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dB || ds)
        CHECK(run_pass(p, p->cols, M_BWD_ROW, vals, B, A, Gn, dB, ds, st));
    if (dA)
        CHECK(run_pass(p, p->rows, M_BWD_COL, vals, A, B, Gn, dA, nullptr, st));
    return FMM_OK;
}

int fmm_plan_status(fmm_plan *p, fmm_stream stream)
{
    CHECK(check_plan(p));
    int32_t flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, p->err, sizeof(flag), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess && flag)
        e = cudaMemsetAsync(p->err, 0, sizeof(int32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("fmm_plan_status", e);
        return FMM_ECUDA;
    }
    if (flag) {
        set_error_msg("a row pass gave up waiting for a gathered row copy");
        return FMM_ETIMEOUT;
    }
    return FMM_OK;
}

const char *fmm_status_string(int status)
{
    switch (status) {
    case FMM_OK: return "ok";
    case FMM_EINVAL: return "invalid argument";
    case FMM_EUNSUPPORTED: return "unsupported";
    case FMM_EOVERFLOW: return "size overflow";
    case FMM_ECUDA: return "CUDA error";
    case FMM_ENOMEM: return "out of device memory";
    case FMM_ETIMEOUT: return "a bounded wait gave up";
    default: return "unknown status";
    }
}

const char *fmm_last_error(void) { return last_error(); }

int32_t fmm_version(void) { return FMM_VERSION; }

}  // extern "C"
