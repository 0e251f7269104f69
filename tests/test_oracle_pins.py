"""Pins of the FP64 oracle against results fixed by the mathematics.

None of these re-types the oracle's loops: each expected value comes from a
different formulation (dense matrix products, closed forms after
re-association, hand arithmetic, finite differences, a transpose built by
scipy) so that a dropped term, a wrong sign or index, or a transposed operand
in oracle/fmm_oracle.c fails at least one of them.

Definitions (Sec. II): SDDMM(A,B,S) = S * (A B^T) (Eq. 1), SpMMA(S,B) = S B,
SpMMB(S,A) = S^T A, FusedMMA = SpMMA(SDDMM, B), FusedMMB = SpMMB(SDDMM, A).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2203_07673_gb300 import workloads as wl


def dense_of(S, vals):
    """Dense m x n matrix of the pattern, duplicates summed (np.add.at)."""
    D = np.zeros((S.m, S.n))
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr.astype(np.int64)))
    v = np.ones(S.nnz) if vals is None else np.asarray(vals, np.float64)
    np.add.at(D, (rows, S.col_idx.astype(np.int64)), v)
    return D


def cases():
    out = []
    for seed, (m, n, r, dup, uns) in enumerate([(7, 5, 3, 0.0, False),
                                                 (33, 17, 8, 0.3, True),
                                                 (64, 64, 16, 0.2, False),
                                                 (1, 40, 5, 0.5, True),
                                                 (40, 1, 4, 0.0, False)]):
        rng = np.random.default_rng(100 + seed)
        S = wl.random_csr(m, n, rng, mean_deg=4, empty_frac=0.25,
                          dup_frac=dup, unsorted=uns)
        vals = rng.uniform(-1, 2, S.nnz)
        A = rng.standard_normal((m, r))
        B = rng.standard_normal((n, r))
        out.append((S, vals, A, B))
    return out


@pytest.mark.parametrize("case", range(5))
def test_bruteforce_dense(case):
    S, vals, A, B = cases()[case]
    D = dense_of(S, vals)
    R = D * (A @ B.T)                      # Eq. (1), dense Hadamard form
    np.testing.assert_allclose(oracle.fusedmm(S.row_ptr, S.col_idx, vals, A, B, S.n),
                               R @ B, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A, B, S.n),
                               R.T @ A, rtol=1e-12, atol=1e-12)
    v = oracle.sddmm(S.row_ptr, S.col_idx, vals, A, B, S.n)
    # scattering the SDDMM values (duplicates summed) gives the dense product
    np.testing.assert_allclose(dense_of(S, v), R, rtol=1e-12, atol=1e-12)
    V = dense_of(S, v)
    np.testing.assert_allclose(oracle.spmm(S.row_ptr, S.col_idx, v, B, S.n),
                               V @ B, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.spmm_t(S.row_ptr, S.col_idx, v, A, S.n),
                               V.T @ A, rtol=1e-12, atol=1e-12)


def test_hand_worked_example():
    # S (2 x 3): s00 = 2, s02 = 1, s11 = 3;  r = 2
    # A = [[1, 2], [0, 1]],  B = [[1, 0], [1, 1], [2, 1]]
    # SDDMM: v00 = 2*<(1,2),(1,0)> = 2;  v02 = 1*<(1,2),(2,1)> = 4;  v11 = 3*<(0,1),(1,1)> = 3
    # FusedMMA: out0 = 2*B0 + 4*B2 = (10, 4);  out1 = 3*B1 = (3, 3)
    # FusedMMB: out0 = 2*A0 = (2, 4);  out1 = 3*A1 = (0, 3);  out2 = 4*A0 = (4, 8)
    rp, ci, s = [0, 2, 3], [0, 2, 1], [2.0, 1.0, 3.0]
    A = np.array([[1.0, 2.0], [0.0, 1.0]])
    B = np.array([[1.0, 0.0], [1.0, 1.0], [2.0, 1.0]])
    assert oracle.sddmm(rp, ci, s, A, B, 3).tolist() == [2.0, 4.0, 3.0]
    assert oracle.fusedmm(rp, ci, s, A, B, 3).tolist() == [[10.0, 4.0], [3.0, 3.0]]
    assert oracle.fusedmm_t(rp, ci, s, A, B, 3).tolist() == [[2.0, 4.0], [0.0, 3.0], [4.0, 8.0]]
    v = [2.0, 4.0, 3.0]
    assert oracle.spmm(rp, ci, v, B, 3).tolist() == [[10.0, 4.0], [3.0, 3.0]]
    assert oracle.spmm_t(rp, ci, v, A, 3).tolist() == [[2.0, 4.0], [0.0, 3.0], [4.0, 8.0]]


def test_all_ones_pattern_closed_form():
    # dense pattern with s = 1: out = (A B^T) B = A (B^T B);  out_t = B (A^T A)
    rng = np.random.default_rng(7)
    m, n, r = 48, 40, 8
    S = wl.CSR(m, n, (np.arange(m + 1) * n).astype(np.int32),
               np.tile(np.arange(n, dtype=np.int32), m))
    A = rng.standard_normal((m, r)); B = rng.standard_normal((n, r))
    np.testing.assert_allclose(oracle.fusedmm(S.row_ptr, S.col_idx, None, A, B, n),
                               A @ (B.T @ B), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(oracle.fusedmm_t(S.row_ptr, S.col_idx, None, A, B, n),
                               B @ (A.T @ A), rtol=1e-11, atol=1e-11)


def test_linearity_and_homogeneity():
    S, vals, A, B = cases()[2]
    rng = np.random.default_rng(3)
    vals2 = rng.uniform(-1, 1, S.nnz)
    F = lambda s, a, b: oracle.fusedmm(S.row_ptr, S.col_idx, s, a, b, S.n)
    Ft = lambda s, a, b: oracle.fusedmm_t(S.row_ptr, S.col_idx, s, a, b, S.n)
    al, be = 0.75, -1.5
    for f in (F, Ft):
        np.testing.assert_allclose(f(al * vals + be * vals2, A, B),
                                   al * f(vals, A, B) + be * f(vals2, A, B),
                                   rtol=1e-11, atol=1e-11)
    # FusedMMA is linear in A and quadratic in B; FusedMMB the other way round
    np.testing.assert_allclose(F(vals, 3 * A, B), 3 * F(vals, A, B), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F(vals, A, -2 * B), 4 * F(vals, A, B), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Ft(vals, -2 * A, B), 4 * Ft(vals, A, B), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Ft(vals, A, 3 * B), 3 * Ft(vals, A, B), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("case", range(5))
def test_transpose_identity(case):
    # FusedMMB(S, A, B) = FusedMMA(S^T, B, A) (Sec. IV-B, last paragraph), with
    # S^T built independently by scipy
    S, vals, A, B = cases()[case]
    M = sp.csr_matrix((vals, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    T = M.T.tocsr()
    lhs = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A, B, S.n)
    rhs = oracle.fusedmm(T.indptr, T.indices, T.data, B, A, S.m)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    lhs = oracle.spmm_t(S.row_ptr, S.col_idx, vals, A, S.n)
    rhs = oracle.spmm(T.indptr, T.indices, T.data, A, S.m)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_special_cases():
    rng = np.random.default_rng(11)
    m, r = 20, 6
    A = rng.standard_normal((m, r)); B = rng.standard_normal((m, r))
    s = rng.uniform(0.5, 2, m)
    eye_rp, eye_ci = np.arange(m + 1), np.arange(m)
    # identity pattern: out_i = s_ii <A_i, B_i> B_i
    exp = (s * np.einsum("ik,ik->i", A, B))[:, None] * B
    np.testing.assert_allclose(oracle.fusedmm(eye_rp, eye_ci, s, A, B, m), exp,
                               rtol=1e-12, atol=1e-12)
    # r = 1: out_i = a_i * sum_j s_ij b_j^2
    S = wl.random_csr(30, 25, rng, mean_deg=5, empty_frac=0.1)
    vals = rng.uniform(-1, 1, S.nnz)
    a = rng.standard_normal((30, 1)); b = rng.standard_normal((25, 1))
    D = dense_of(S, vals)
    np.testing.assert_allclose(oracle.fusedmm(S.row_ptr, S.col_idx, vals, a, b, 25),
                               a * (D @ (b[:, 0] ** 2))[:, None], rtol=1e-12, atol=1e-12)
    # one nonzero: the SDDMM is a plain dot product
    x = rng.standard_normal((1, 9)); y = rng.standard_normal((3, 9))
    v = oracle.sddmm([0, 1], [2], [1.0], x, y, 3)
    assert v[0] == pytest.approx(float(np.dot(x[0], y[2])), rel=1e-14)
    # empty S and empty shapes give zeros
    z = oracle.fusedmm(np.zeros(6, np.int64), [], None, np.ones((5, 3)), np.ones((4, 3)), 4)
    assert z.shape == (5, 3) and not z.any()
    zt = oracle.fusedmm_t(np.zeros(6, np.int64), [], None, np.ones((5, 3)), np.ones((4, 3)), 4)
    assert zt.shape == (4, 3) and not zt.any()
    assert oracle.fusedmm([0], [], None, np.ones((0, 3)), np.ones((4, 3)), 4).shape == (0, 3)


def test_malformed_csr_rejected():
    with pytest.raises(ValueError):
        oracle.fusedmm([0, 1], [5], None, np.ones((1, 2)), np.ones((3, 2)), 3)
    with pytest.raises(ValueError):
        oracle.sddmm([0, 2, 1], [0, 0], None, np.ones((2, 2)), np.ones((3, 2)), 3)


def test_exact_small_integers():
    # |x| <= 4, r <= 16, degree <= 32: every partial sum is an exact integer
    rng = np.random.default_rng(5)
    S = wl.random_csr(50, 37, rng, mean_deg=10, empty_frac=0.1, dup_frac=0.2)
    vals = wl.small_ints(S.nnz, 4, rng).astype(np.float64)
    A = wl.small_ints((50, 16), 4, rng).astype(np.float64)
    B = wl.small_ints((37, 16), 4, rng).astype(np.float64)
    R = dense_of(S, vals) * (A @ B.T)
    assert np.array_equal(oracle.fusedmm(S.row_ptr, S.col_idx, vals, A, B, 37), R @ B)
    assert np.array_equal(oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A, B, 37), R.T @ A)


def _fd_grad(f, x, h=1e-6):
    g = np.zeros_like(x)
    flat, gf = x.reshape(-1), g.reshape(-1)
    for t in range(flat.size):
        old = flat[t]
        flat[t] = old + h; fp = f()
        flat[t] = old - h; fm = f()
        flat[t] = old
        gf[t] = (fp - fm) / (2 * h)
    return g


@pytest.mark.parametrize("transpose", [False, True])
def test_gradient_finite_differences(transpose):
    rng = np.random.default_rng(21 + transpose)
    S = wl.random_csr(9, 7, rng, mean_deg=3, empty_frac=0.2, dup_frac=0.2)
    r = 4
    vals = rng.uniform(-1, 1, S.nnz)
    A = rng.standard_normal((9, r)); B = rng.standard_normal((7, r))
    G = rng.standard_normal((7 if transpose else 9, r))
    fwd = oracle.fusedmm_t if transpose else oracle.fusedmm
    grad = oracle.fusedmm_t_grad if transpose else oracle.fusedmm_grad
    L = lambda: float(np.sum(G * fwd(S.row_ptr, S.col_idx, vals, A, B, 7)))
    dA, dB, ds = grad(S.row_ptr, S.col_idx, vals, A, B, G, 7)
    for analytic, x in ((dA, A), (dB, B), (ds, vals)):
        fd = _fd_grad(L, x)
        err = np.linalg.norm(fd - analytic) / max(np.linalg.norm(analytic), 1e-300)
        assert err <= 1e-6, err


def test_gradient_dense_closed_form():
    # L = <G, (S o (A B^T)) B>: dA = (S o (G B^T)) B,
    # dB = (S o (A B^T))^T G + (S o (G B^T))^T A,  ds_ij = (A B^T)_ij (G B^T)_ij
    S, vals, A, B = cases()[2]
    # distinct entries only, so each nonzero's ds can be read from a dense matrix
    M = sp.csr_matrix((vals, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    M.sum_duplicates()
    rp, ci, vv = M.indptr, M.indices, M.data
    rng = np.random.default_rng(9)
    G = rng.standard_normal((S.m, A.shape[1]))
    D = M.toarray()
    dA, dB, ds = oracle.fusedmm_grad(rp, ci, vv, A, B, G, S.n)
    np.testing.assert_allclose(dA, (D * (G @ B.T)) @ B, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dB, (D * (A @ B.T)).T @ G + (D * (G @ B.T)).T @ A,
                               rtol=1e-11, atol=1e-11)
    rows = np.repeat(np.arange(S.m), np.diff(rp))
    np.testing.assert_allclose(ds, (A @ B.T)[rows, ci] * (G @ B.T)[rows, ci],
                               rtol=1e-11, atol=1e-11)
    # FusedMMB: L = <Gn, (S o (A B^T))^T A>
    Gn = rng.standard_normal((S.n, A.shape[1]))
    dA, dB, ds = oracle.fusedmm_t_grad(rp, ci, vv, A, B, Gn, S.n)
    W = D * (A @ Gn.T)
    np.testing.assert_allclose(dB, W.T @ A, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dA, (D * (A @ B.T)) @ Gn + W @ B, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(ds, (A @ B.T)[rows, ci] * (A @ Gn.T)[rows, ci],
                               rtol=1e-11, atol=1e-11)


def test_golden_fixture():
    # regression fixture written by tests/golden/make_golden.py (oracle only)
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    make_golden = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(make_golden)
    fx = make_golden.read(os.path.join(here, "fusedmm_small.txt"))
    out = oracle.fusedmm(fx["row_ptr"], fx["col_idx"], fx["vals"], fx["A"], fx["B"], fx["n"])
    out_t = oracle.fusedmm_t(fx["row_ptr"], fx["col_idx"], fx["vals"], fx["A"], fx["B"], fx["n"])
    np.testing.assert_allclose(out, fx["out"], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(out_t, fx["out_t"], rtol=1e-15, atol=1e-15)
