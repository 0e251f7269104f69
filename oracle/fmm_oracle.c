/*
 * FP64 CPU oracle for FusedMM: an SDDMM feeding an SpMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or run this code; the
 * product library (libfmm) never calls it, and the two share no source,
 * header, helper or table.
 *
 * Every routine is the plain definition written out as loops, in FP64, with
 * the inner product summed over k in ascending order and the nonzeros of a
 * row visited in CSR order.  No blocking, no reordering, no fusion beyond
 * what the definition itself states.
 *
 * Sparse S is given as CSR with 64-bit row pointers and column indices:
 *   rowptr[m+1], colidx[nnz], vals[nnz] (vals == NULL means every s_ij = 1).
 * Dense matrices are row-major: A is m x r, B is n x r, G is m x r (or n x r).
 * Duplicate (i, j) entries are allowed and each one contributes; columns of a
 * row need not be sorted.
 *
 * Each routine returns 0, or -1 if an index is outside its matrix (the
 * outputs are then unspecified).
 *
 * Paper passages followed (Bharadwaj, Buluc, Demmel, "Distributed-Memory
 * Sparse Kernels for Machine Learning"):
 *   Sec. II, Eq. (1)        SDDMM(A, B, S) = S * (A B^T), only at nonzeros of S
 *   Sec. II                 SpMMA(S, B) = S B,  SpMMB(S, A) = S^T A,
 *                           FusedMMA = SpMMA(SDDMM(A,B,S), B),
 *                           FusedMMB = SpMMB(SDDMM(A,B,S), A)
 *   Sec. IV-A               per-nonzero SpMMA update A_i += S_ij B_j
 *   Sec. IV-B               row form FusedMMA_i = sum_j S_ij <A_i, B_j> B_j
 *   Sec. VI-E               ALS: per-row least squares M x = b solved by CG,
 *                           the queries M x batched as FusedMM; GAT: the
 *                           attention variant of SDDMM, softmax, aggregation
 * The gradients are not in the paper; they are the derivatives of the
 * scalar L = <G, FusedMM(S, A, B)> with respect to A, B and the values of S,
 * on a fixed pattern.
 *
 * Built as a shared library by oracle/build.py:
 *   gcc -O2 -fopenmp -fPIC -shared -lm -o oracle/_build/liboracle.so oracle/fmm_oracle.c
 * Rows are independent in the row-wise routines, so those loop over rows with
 * an OpenMP parallel-for; the scatter routines run sequentially.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double oracle_s(const double *vals, int64_t p)
{
    return vals ? vals[p] : 1.0;
}

/* <x, y> = sum_{k < r} x[k] * y[k], k ascending. */
static double oracle_dot(const double *x, const double *y, int64_t r)
{
    double acc = 0.0;
    for (int64_t k = 0; k < r; ++k)
        acc += x[k] * y[k];
    return acc;
}

static int oracle_check(int64_t m, int64_t n, const int64_t *rowptr,
                        const int64_t *colidx)
{
    if (m < 0 || n < 0 || rowptr[0] != 0)
        return -1;
    for (int64_t i = 0; i < m; ++i) {
        if (rowptr[i + 1] < rowptr[i])
            return -1;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (colidx[p] < 0 || colidx[p] >= n)
                return -1;
    }
    return 0;
}

/* SDDMM, Sec. II Eq. (1): v[p] = s_ij * <A_i, B_j> for the p-th nonzero (i, j). */
int oracle_sddmm(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                 const int64_t *colidx, const double *vals, const double *A,
                 const double *B, double *v)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            v[p] = oracle_s(vals, p) * oracle_dot(A + i * r, B + j * r, r);
        }
    return 0;
}

/* SpMMA, Sec. II and the update of Sec. IV-A: out_i = sum_p v[p] * B_j. */
int oracle_spmm(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                const int64_t *colidx, const double *v, const double *B,
                double *out)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *o = out + i * r;
        for (int64_t k = 0; k < r; ++k)
            o[k] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double *b = B + colidx[p] * r;
            for (int64_t k = 0; k < r; ++k)
                o[k] += v[p] * b[k];
        }
    }
    return 0;
}

/* SpMMB, Sec. II: out = S^T A, i.e. out_j += v[p] * A_i for each nonzero
 * (i, j), scattered straight from the CSR of S (no transposed copy). */
int oracle_spmm_t(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                  const int64_t *colidx, const double *v, const double *A,
                  double *out)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    memset(out, 0, (size_t)(n * r) * sizeof(double));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double *o = out + colidx[p] * r;
            const double *a = A + i * r;
            for (int64_t k = 0; k < r; ++k)
                o[k] += v[p] * a[k];
        }
    return 0;
}

/* FusedMMA, Sec. II and its row form in Sec. IV-B:
 * out_i = sum_{(i,j) in nnz(S)} s_ij <A_i, B_j> B_j.
 * The SDDMM value of each nonzero is held in one scalar and used at once. */
int oracle_fusedmm(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                   const int64_t *colidx, const double *vals, const double *A,
                   const double *B, double *out)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *o = out + i * r;
        for (int64_t k = 0; k < r; ++k)
            o[k] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double *b = B + colidx[p] * r;
            double v = oracle_s(vals, p) * oracle_dot(A + i * r, b, r);
            for (int64_t k = 0; k < r; ++k)
                o[k] += v * b[k];
        }
    }
    return 0;
}

/* FusedMMB, Sec. II: out = S'^T A with S' = SDDMM(A, B, S), i.e.
 * out_j = sum_{(i,j) in nnz(S)} s_ij <A_i, B_j> A_i.
 * Scattered directly over the CSR of S; deliberately builds no S^T. */
int oracle_fusedmm_t(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                     const int64_t *colidx, const double *vals, const double *A,
                     const double *B, double *out)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    memset(out, 0, (size_t)(n * r) * sizeof(double));
    for (int64_t i = 0; i < m; ++i) {
        const double *a = A + i * r;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            double v = oracle_s(vals, p) * oracle_dot(a, B + j * r, r);
            double *o = out + j * r;
            for (int64_t k = 0; k < r; ++k)
                o[k] += v * a[k];
        }
    }
    return 0;
}

/* Gradient of L = sum_i <G_i, FusedMMA(S, A, B)_i> (G is m x r).
 * With d = <A_i, B_j> and w = <G_i, B_j> at nonzero p = (i, j):
 *   ds[p] = d * w
 *   dA_i  = sum_p s_ij * w * B_j
 *   dB_j  = sum_p s_ij * (d * G_i + w * A_i)
 * Any of dA, dB, ds may be NULL.  Sequential (dB is a scatter). */
int oracle_fusedmm_grad(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                        const int64_t *colidx, const double *vals,
                        const double *A, const double *B, const double *G,
                        double *dA, double *dB, double *ds)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    if (dA)
        memset(dA, 0, (size_t)(m * r) * sizeof(double));
    if (dB)
        memset(dB, 0, (size_t)(n * r) * sizeof(double));
    for (int64_t i = 0; i < m; ++i) {
        const double *a = A + i * r, *g = G + i * r;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            const double *b = B + j * r;
            double s = oracle_s(vals, p);
            double d = oracle_dot(a, b, r);
            double w = oracle_dot(g, b, r);
            if (ds)
                ds[p] = d * w;
            if (dA)
                for (int64_t k = 0; k < r; ++k)
                    dA[i * r + k] += s * w * b[k];
            if (dB)
                for (int64_t k = 0; k < r; ++k)
                    dB[j * r + k] += s * (d * g[k] + w * a[k]);
        }
    }
    return 0;
}

/* Gradient of L = sum_j <Gn_j, FusedMMB(S, A, B)_j> (Gn is n x r).
 * With d = <A_i, B_j> and w = <Gn_j, A_i> at nonzero p = (i, j):
 *   ds[p] = d * w
 *   dB_j  = sum_p s_ij * w * A_i
 *   dA_i  = sum_p s_ij * (d * Gn_j + w * B_j)
 * Any of dA, dB, ds may be NULL.  Sequential. */
int oracle_fusedmm_t_grad(int64_t m, int64_t n, int64_t r,
                          const int64_t *rowptr, const int64_t *colidx,
                          const double *vals, const double *A, const double *B,
                          const double *Gn, double *dA, double *dB, double *ds)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    if (dA)
        memset(dA, 0, (size_t)(m * r) * sizeof(double));
    if (dB)
        memset(dB, 0, (size_t)(n * r) * sizeof(double));
    for (int64_t i = 0; i < m; ++i) {
        const double *a = A + i * r;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int64_t j = colidx[p];
            const double *b = B + j * r, *g = Gn + j * r;
            double s = oracle_s(vals, p);
            double d = oracle_dot(a, b, r);
            double w = oracle_dot(g, a, r);
            if (ds)
                ds[p] = d * w;
            if (dB)
                for (int64_t k = 0; k < r; ++k)
                    dB[j * r + k] += s * w * a[k];
            if (dA)
                for (int64_t k = 0; k < r; ++k)
                    dA[i * r + k] += s * (d * g[k] + w * b[k]);
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * ALS with conjugate gradients (Sec. VI-E, collaborative filtering).
 *
 * The loss is the squared Frobenius norm of (C - SDDMM(A, B, S)) over the
 * nonzeros of S, plus lambda (|A|^2 + |B|^2).  With B fixed, each row A_i
 * solves the normal equations M_i x = b_i,
 *     M_i x = sum_{j in row i} <x, B_j> B_j + lambda x,   b_i = sum_j c_ij B_j,
 * and with A fixed each row B_j solves the same with the roles exchanged
 * (the sum running over the nonzeros of column j).  M_i x for all rows at
 * once is FusedMMA of the 0/1 pattern (FusedMMB for the B side), as the
 * paper batches the CG queries.  This routine runs `iters` plain CG
 * iterations per row, started from the current rows, in FP64:
 *     r = b - M x;  p = r;  rs = <r, r>
 *     repeat: q = M p;  alpha = rs / <p, q>;  x += alpha p;  r -= alpha q;
 *             rs' = <r, r>;  p = r + (rs' / rs) p;  rs = rs'
 * with alpha = 0 when <p, q> <= 0 and the ratio 0 when rs = 0.
 * side 0 updates A (m x r, in place); side 1 updates B (n x r, in place).
 * c: nnz values in CSR order.  Sequential.
 * ------------------------------------------------------------------------ */
static void oracle_apply_m(int64_t r, double lambda, int64_t deg, const int64_t *nbr,
                           const double *Y, const double *x, double *out)
{
    for (int64_t k = 0; k < r; ++k)
        out[k] = lambda * x[k];
    for (int64_t t = 0; t < deg; ++t) {
        const double *y = Y + nbr[t] * r;
        double d = oracle_dot(x, y, r);
        for (int64_t k = 0; k < r; ++k)
            out[k] += d * y[k];
    }
}

/* The CG of every row of one side, with its state exposed.  When init is
 * set the state starts from the current rows:  r = b - M x;  p = r;
 * rs = <r, r>;  otherwise res, p (rows x r) and rs (rows) hold the state
 * of an earlier call.  Then `iters` iterations as above.  res, p and rs
 * may be NULL when init is set (the state is then kept internally and
 * dropped on return). */
static int oracle_als_cg_core(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                              const int64_t *colidx, const double *c, double *A, double *B,
                              double lambda, int64_t iters, int side, int init,
                              double *res_io, double *p_io, double *rs_io)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    if (!init && (!res_io || !p_io || !rs_io))
        return -1;
    int64_t nnz = rowptr[m];
    /* neighbour lists of every row of the side being updated */
    int64_t rows = side == 0 ? m : n;
    int64_t *start = calloc((size_t)rows + 1, sizeof(int64_t));
    int64_t *nbr = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    double *cv = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    double *w = malloc((size_t)(4 * r > 0 ? 4 * r : 1) * sizeof(double));
    if (!start || !nbr || !cv || !w) {
        free(start); free(nbr); free(cv); free(w);
        return -2;
    }
    if (side == 0) {
        for (int64_t i = 0; i <= m; ++i)
            start[i] = rowptr[i];
        for (int64_t p = 0; p < nnz; ++p) {
            nbr[p] = colidx[p];
            cv[p] = c ? c[p] : 0.0;
        }
    } else {
        for (int64_t p = 0; p < nnz; ++p)
            start[colidx[p] + 1]++;
        for (int64_t j = 0; j < n; ++j)
            start[j + 1] += start[j];
        int64_t *fill = calloc((size_t)n, sizeof(int64_t));
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int64_t j = colidx[p];
                int64_t q = start[j] + fill[j]++;
                nbr[q] = i;
                cv[q] = c ? c[p] : 0.0;
            }
        free(fill);
    }
    double *X = side == 0 ? A : B;
    const double *Y = side == 0 ? B : A;
    double *q = w + 2 * r, *bb = w + 3 * r;
    for (int64_t i = 0; i < rows; ++i) {
        int64_t deg = start[i + 1] - start[i];
        const int64_t *nb = nbr + start[i];
        double *x = X + i * r;
        double *res = res_io ? res_io + i * r : w;
        double *pp = p_io ? p_io + i * r : w + r;
        double rs;
        if (init) {
            for (int64_t k = 0; k < r; ++k)
                bb[k] = 0.0;
            for (int64_t t = 0; t < deg; ++t)
                for (int64_t k = 0; k < r; ++k)
                    bb[k] += cv[start[i] + t] * Y[nb[t] * r + k];
            oracle_apply_m(r, lambda, deg, nb, Y, x, q);
            for (int64_t k = 0; k < r; ++k) {
                res[k] = bb[k] - q[k];
                pp[k] = res[k];
            }
            rs = oracle_dot(res, res, r);
        } else {
            rs = rs_io[i];
        }
        for (int64_t it = 0; it < iters; ++it) {
            oracle_apply_m(r, lambda, deg, nb, Y, pp, q);
            double pq = oracle_dot(pp, q, r);
            double alpha = pq > 0.0 ? rs / pq : 0.0;
            for (int64_t k = 0; k < r; ++k) {
                x[k] += alpha * pp[k];
                res[k] -= alpha * q[k];
            }
            double rs2 = oracle_dot(res, res, r);
            double beta = rs > 0.0 ? rs2 / rs : 0.0;
            for (int64_t k = 0; k < r; ++k)
                pp[k] = res[k] + beta * pp[k];
            rs = rs2;
        }
        if (rs_io)
            rs_io[i] = rs;
    }
    free(start); free(nbr); free(cv); free(w);
    return 0;
}

int oracle_als_cg(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                  const int64_t *colidx, const double *c, double *A, double *B,
                  double lambda, int64_t iters, int side)
{
    return oracle_als_cg_core(m, n, r, rowptr, colidx, c, A, B, lambda, iters, side, 1,
                              NULL, NULL, NULL);
}

/* The same CG with its state in the caller's arrays: init = 1 starts from
 * the current rows (c is read) and writes the state after `iters`
 * iterations into res, p (rows x r) and rs (rows); init = 0 continues from
 * the state given there (c is not read and may be NULL). */
int oracle_als_cg_state(int64_t m, int64_t n, int64_t r, const int64_t *rowptr,
                        const int64_t *colidx, const double *c, double *A, double *B,
                        double lambda, int64_t iters, int side, int init, double *res,
                        double *p, double *rs)
{
    if (!res || !p || !rs)
        return -1;
    return oracle_als_cg_core(m, n, r, rowptr, colidx, c, A, B, lambda, iters, side, init,
                              res, p, rs);
}

/* ---------------------------------------------------------------------------
 * Graph-attention layer, forward (Sec. VI-E, GAT workload).
 *
 * One attention head replaces S by S' = LeakyReLU(S * (H .GAT H^T)) with
 * (H .GAT H^T)_ij = a^T (H_i || H_j) = a_l^T H_i + a_r^T H_j, normalises each
 * row of S' with a softmax over its nonzeros and aggregates the rows of H:
 *     e_ij  = LeakyReLU(s_ij * (f_i + g_j)),  f = H_dst a_l,  g = H a_r
 *     alpha = softmax over the nonzeros of row i of e_ij
 *     out_i = sum_j alpha_ij H_j
 * Multi-head: `heads` independent heads, head h using columns
 * [h * rh, (h + 1) * rh) of H (n x heads*rh) and out (m x heads*rh), and
 * f[i * heads + h], g[j * heads + h].  LeakyReLU(x) = x if x > 0 else
 * slope * x.  Rows without nonzeros give zeros.  Softmax in the textbook
 * two-pass form: max, then sum of exp(e - max).  Rows in parallel.
 * ------------------------------------------------------------------------ */
#include <math.h>

int oracle_gat(int64_t m, int64_t n, int64_t heads, int64_t rh, const int64_t *rowptr,
               const int64_t *colidx, const double *vals, const double *f, const double *g,
               const double *H, double slope, double *out)
{
    if (oracle_check(m, n, rowptr, colidx))
        return -1;
    const int64_t r = heads * rh;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = 0; k < r; ++k)
            out[i * r + k] = 0.0;
        for (int64_t h = 0; h < heads; ++h) {
            double mx = -INFINITY;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                double x = oracle_s(vals, p) * (f[i * heads + h] + g[colidx[p] * heads + h]);
                double e = x > 0.0 ? x : slope * x;
                if (e > mx)
                    mx = e;
            }
            double sum = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                double x = oracle_s(vals, p) * (f[i * heads + h] + g[colidx[p] * heads + h]);
                double e = x > 0.0 ? x : slope * x;
                sum += exp(e - mx);
            }
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                double x = oracle_s(vals, p) * (f[i * heads + h] + g[colidx[p] * heads + h]);
                double e = x > 0.0 ? x : slope * x;
                double a = exp(e - mx) / sum;
                const double *hj = H + colidx[p] * r + h * rh;
                for (int64_t k = 0; k < rh; ++k)
                    out[i * r + h * rh + k] += a * hj[k];
            }
        }
    }
    return 0;
}

/* Thread count of the row loops (timing of the CPU baseline only): sets it
 * when n > 0, and returns the number of threads a parallel row loop uses. */
#ifdef _OPENMP
#include <omp.h>
#endif
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
