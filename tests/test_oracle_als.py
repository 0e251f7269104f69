"""Pins of the oracle's ALS-CG routine (Sec. VI-E) against closed forms.

Each row solves (sum_j B_j B_j^T + lam I) x = sum_j c_ij B_j.  CG on an
r-dimensional SPD system reaches the exact solution in r iterations (exact
arithmetic), so after r iterations the oracle must match a dense solve built
here with numpy; one iteration from zero has the closed form
x = (b.b / b.M b) b; the B side equals the A side on the transposed pattern.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2203_07673_gb300 import workloads as wl


def _problem(seed, m=40, n=30, r=4):
    rng = np.random.default_rng(seed)
    S = wl.random_csr(m, n, rng, mean_deg=5, empty_frac=0.1)
    c = rng.uniform(1, 5, S.nnz)
    A = rng.standard_normal((m, r))
    B = rng.standard_normal((n, r))
    return S, c, A, B


def _dense_solution(S, c, A, B, lam, side):
    M = sp.csr_matrix((c, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    P = sp.csr_matrix((np.ones(S.nnz), S.col_idx, S.row_ptr), shape=(S.m, S.n))
    if side == 1:
        M, P, A, B = M.T.tocsr(), P.T.tocsr(), B, A
    r = A.shape[1]
    X = np.zeros_like(A)
    for i in range(A.shape[0]):
        nb = P.indices[P.indptr[i]:P.indptr[i + 1]]
        cv = M.data[M.indptr[i]:M.indptr[i + 1]] if M.nnz else np.zeros(0)
        Mi = B[nb].T @ B[nb] + lam * np.eye(r)
        bi = B[nb].T @ cv
        X[i] = np.linalg.solve(Mi, bi)
    return X


@pytest.mark.parametrize("side", [0, 1])
def test_cg_reaches_the_dense_solution_in_r_iterations(side):
    S, c, A, B = _problem(1 + side)
    lam = 0.5
    exact = _dense_solution(S, c, A, B, lam, side)
    got = oracle.als_cg(S.row_ptr, S.col_idx, c, A, B, lam, A.shape[1], side)
    np.testing.assert_allclose(got, exact, rtol=1e-7, atol=1e-9)


def test_one_iteration_from_zero_closed_form():
    S, c, A, B = _problem(3)
    lam = 0.25
    got = oracle.als_cg(S.row_ptr, S.col_idx, c, np.zeros_like(A), B, lam, 1, 0)
    for i in range(S.m):
        nb = S.col_idx[S.row_ptr[i]:S.row_ptr[i + 1]]
        cv = c[S.row_ptr[i]:S.row_ptr[i + 1]]
        b = B[nb].T @ cv
        Mb = B[nb].T @ (B[nb] @ b) + lam * b
        den = b @ Mb
        exp = (b @ b) / den * b if den > 0 else np.zeros_like(b)
        np.testing.assert_allclose(got[i], exp, rtol=1e-12, atol=1e-14)


def test_b_side_equals_a_side_on_the_transpose():
    S, c, A, B = _problem(4)
    M = sp.csr_matrix((c, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    T = M.T.tocsr()
    got = oracle.als_cg(S.row_ptr, S.col_idx, c, A, B, 0.3, 3, 1)
    exp = oracle.als_cg(T.indptr, T.indices, T.data, B, A, 0.3, 3, 0)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-12)


def test_als_loss_decreases():
    S, c, A, B = _problem(5, m=60, n=50, r=6)
    lam = 0.1

    def loss(A, B):
        rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
        pred = np.einsum("ij,ij->i", A[rows], B[S.col_idx])
        return np.sum((c - pred) ** 2) + lam * (np.sum(A * A) + np.sum(B * B))

    prev = loss(A, B)
    for _ in range(3):
        A = oracle.als_cg(S.row_ptr, S.col_idx, c, A, B, lam, 6, 0)
        cur = loss(A, B)
        assert cur <= prev + 1e-9
        prev = cur
        B = oracle.als_cg(S.row_ptr, S.col_idx, c, A, B, lam, 6, 1)
        cur = loss(A, B)
        assert cur <= prev + 1e-9
        prev = cur


def _rows_of_side(S, c, A, B, side):
    """Per row of the side: (neighbour rows of the fixed factor, observations)."""
    M = sp.csr_matrix((c, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    if side == 1:
        M, A, B = M.T.tocsr(), B, A
    P = sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape)
    out = []
    for i in range(M.shape[0]):
        nb = P.indices[P.indptr[i]:P.indptr[i + 1]]
        out.append((nb, M.data[M.indptr[i]:M.indptr[i + 1]]))
    return out, A, B


@pytest.mark.parametrize("side", [0, 1])
def test_cg_state_after_init_is_the_residual(side):
    """init: res = b - (Y^T Y + lam I) x with b = Y^T c, p = res, rs = |res|^2,
    built per row from dense products."""
    S, c, A, B = _problem(6 + side)
    lam = 0.4
    X, res, p, rs = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, lam, 0, side)
    rows, Xin, Y = _rows_of_side(S, c, A, B, side)
    np.testing.assert_array_equal(X, Xin)
    for i, (nb, cv) in enumerate(rows):
        Mi = Y[nb].T @ Y[nb] + lam * np.eye(Y.shape[1])
        exp = Y[nb].T @ cv - Mi @ Xin[i]
        np.testing.assert_allclose(res[i], exp, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(p[i], res[i])
        np.testing.assert_allclose(rs[i], exp @ exp, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("side", [0, 1])
def test_cg_steps_from_passed_state_reach_the_dense_solution(side):
    """r single iterations, each continuing from the state the previous call
    returned, solve every row's r x r system exactly (exact arithmetic): the
    state (res, p, rs) is carried between calls correctly."""
    S, c, A, B = _problem(8 + side)
    lam = 0.5
    exact = _dense_solution(S, c, A, B, lam, side)
    X, res, p, rs = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, lam, 0, side)
    for _ in range(A.shape[1]):
        Ain, Bin = (X, B) if side == 0 else (A, X)
        X, res, p, rs = oracle.als_cg_state(S.row_ptr, S.col_idx, None, Ain, Bin, lam, 1, side,
                                            state=(res, p, rs))
    np.testing.assert_allclose(X, exact, rtol=1e-7, atol=1e-9)


def test_one_step_from_state_closed_form():
    """From x = 0 (res = p = b, rs = |b|^2) one iteration gives
    alpha = |b|^2 / b^T M b, x = alpha b, res = b - alpha M b,
    p = res + (|res|^2 / |b|^2) b."""
    S, c, A, B = _problem(10)
    lam = 0.3
    rows, _, Y = _rows_of_side(S, c, A, B, 0)
    b = np.zeros_like(A)
    for i, (nb, cv) in enumerate(rows):
        b[i] = Y[nb].T @ cv
    rs0 = np.einsum("ij,ij->i", b, b)
    X, res, p, rs = oracle.als_cg_state(S.row_ptr, S.col_idx, None, np.zeros_like(A), B, lam,
                                        1, 0, state=(b, b, rs0))
    for i, (nb, _) in enumerate(rows):
        Mb = Y[nb].T @ (Y[nb] @ b[i]) + lam * b[i]
        den = b[i] @ Mb
        alpha = rs0[i] / den if den > 0 else 0.0
        res_e = b[i] - alpha * Mb
        rs_e = res_e @ res_e
        p_e = res_e + (rs_e / rs0[i] if rs0[i] > 0 else 0.0) * b[i]
        np.testing.assert_allclose(X[i], alpha * b[i], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(res[i], res_e, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(p[i], p_e, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(rs[i], rs_e, rtol=1e-10, atol=1e-14)
