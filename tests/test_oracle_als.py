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
