"""CPU checks of the element-wise bounds that the GPU ALS test applies
(tests/als_bounds.py; ALS with CG, Sec. VI-E).

1. The bounds admit float32 arithmetic: the same CG steps computed in float32
   with numpy/scipy (another summation order than the GPU's) stay within them.
2. They reject a wrong regulariser.  The mistake is planted in the oracle: the
   oracle's step is rerun with a wrong lambda and one row of its result is
   spliced into the correct one; the comparison must fail for a dropped
   lambda on the split hub row (400 nonzeros), a doubled lambda and a lambda
   off by 1 % on an ordinary row, and a dropped lambda in the set-up.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import als_bounds as ab
import oracle
from paper_2203_07673_gb300 import workloads as wl

F32 = np.float32


def _problem(seed, m=300, n=220, r=32):
    rng = np.random.default_rng(seed)
    S = wl.random_csr(m, n, rng, mean_deg=10, empty_frac=0.05, hubs=((3, 400),))
    c = wl.half_steps(S.nnz, 1.0, 5.0, rng)
    A = (rng.standard_normal((m, r)) * 0.3).astype(np.float32)
    B = (rng.standard_normal((n, r)) * 0.3).astype(np.float32)
    return S, c.astype(np.float32), A, B


def _fusedmm32(S, side, X, Y):
    rows_of = np.repeat(np.arange(S.m), np.diff(S.row_ptr.astype(np.int64)))
    if side == 0:
        d = np.einsum("ij,ij->i", X[rows_of], Y[S.col_idx]).astype(F32)
        M = sp.csr_matrix((d, S.col_idx, S.row_ptr), shape=(S.m, S.n))
        return (M @ Y).astype(F32)
    d = np.einsum("ij,ij->i", Y[rows_of], X[S.col_idx]).astype(F32)
    M = sp.csr_matrix((d, S.col_idx, S.row_ptr), shape=(S.m, S.n)).T.tocsr()
    return (M @ Y).astype(F32)


def _spmm32(S, side, c, Y):
    M = sp.csr_matrix((c, S.col_idx, S.row_ptr), shape=(S.m, S.n))
    if side == 1:
        M = M.T.tocsr()
    return (M @ Y).astype(F32)


def _init32(S, side, c, X, Y, lam):
    b = _spmm32(S, side, c, Y)
    q = _fusedmm32(S, side, X, Y)
    res = (b - q - F32(lam) * X).astype(F32)
    return res, res.copy(), (res * res).sum(1, dtype=F32)


def _step32(S, side, X, res, p, rs, Y, lam):
    q = _fusedmm32(S, side, p, Y)
    t = (q + F32(lam) * p).astype(F32)
    pt = (p * t).sum(1, dtype=F32)
    with np.errstate(divide="ignore", invalid="ignore"):
        alpha = np.where(pt > 0, rs / pt, 0).astype(F32)[:, None]
    X = (X + alpha * p).astype(F32)
    res = (res - alpha * t).astype(F32)
    rr = (res * res).sum(1, dtype=F32)
    with np.errstate(divide="ignore", invalid="ignore"):
        beta = np.where(rs > 0, rr / rs, 0).astype(F32)[:, None]
    return X, res, (res + beta * p).astype(F32), rr


def _w64(*xs):
    return [np.asarray(x, np.float64) for x in xs]


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("r", [32, 64])
def test_float32_cg_steps_stay_within_the_bounds(r, side):
    S, c, A, B = _problem(r + side, r=r)
    lam = 1.0
    X = (A if side == 0 else B).copy()
    Y = B if side == 0 else A
    res, p, rs = _init32(S, side, c, X, Y, lam)
    _, res_o, _, rs_o = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, lam, 0, side)
    dres, drs = ab.init_bound(S, side, *_w64(c, X, Y), lam, r)
    assert ab.check("res", res, res_o, dres) < 0.5
    assert ab.check("rs", rs, rs_o, drs) < 0.5
    for _ in range(3):
        st = _w64(X, res, p, rs)
        X, res, p, rs = _step32(S, side, X, res, p, rs, Y, lam)
        Ain, Bin = (st[0], B) if side == 0 else (A, st[0])
        ref = oracle.als_cg_state(S.row_ptr, S.col_idx, None, Ain, Bin, lam, 1, side,
                                  state=st[1:])
        bnd = ab.step_bound(S, side, *st, np.asarray(Y, np.float64), lam, r)
        for name, got, o, b in zip(("x", "res", "p", "rs"), (X, res, p, rs), ref, bnd):
            assert ab.check(name, got, o, b) < 0.5


def _step_rejects(S, c, side, A, B, lam, row, lam_wrong, r):
    """Whether the step comparison rejects the oracle's step with lam_wrong
    on `row` (every other row correct)."""
    _, res0, p0, rs0 = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, lam, 0, side)
    X0 = np.asarray(A if side == 0 else B, np.float64)
    Y = np.asarray(B if side == 0 else A, np.float64)
    st = [X0] + [np.float32(x).astype(np.float64) for x in (res0, p0, rs0)]
    Ain, Bin = (st[0], B) if side == 0 else (A, st[0])
    good = oracle.als_cg_state(S.row_ptr, S.col_idx, None, Ain, Bin, lam, 1, side, state=st[1:])
    bad = oracle.als_cg_state(S.row_ptr, S.col_idx, None, Ain, Bin, lam_wrong, 1, side,
                              state=st[1:])
    bnd = ab.step_bound(S, side, *st, Y, lam, r)
    for name, g, w, b in zip(("x", "res", "p", "rs"), good, bad, bnd):
        mut = g.copy()
        mut[row] = w[row]
        try:
            ab.check(name, mut, g, b)
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("r", [32, 64])
def test_wrong_lambda_is_rejected(r):
    S, c, A, B = _problem(7 + r, r=r)
    lam = 1.0
    deg = ab.side_degrees(S, 0)
    hub = int(np.argmax(deg))
    assert deg[hub] >= 400
    ordinary = int(np.nonzero((deg > 0) & (deg < 40))[0][0])
    assert _step_rejects(S, c, 0, A, B, lam, hub, 0.0, r), "dropped lambda on the hub row"
    assert _step_rejects(S, c, 0, A, B, lam, ordinary, 2.0 * lam, r), "doubled lambda"
    assert _step_rejects(S, c, 0, A, B, lam, ordinary, 1.01 * lam, r), "lambda off by 1 %"
    assert not _step_rejects(S, c, 0, A, B, lam, ordinary, lam, r), "the correct step"
    # the set-up with lambda dropped on the hub row
    _, res_ok, _, _ = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, lam, 0, 0)
    _, res_bad, _, _ = oracle.als_cg_state(S.row_ptr, S.col_idx, c, A, B, 0.0, 0, 0)
    mut = res_ok.copy()
    mut[hub] = res_bad[hub]
    dres, _ = ab.init_bound(S, 0, *_w64(c, A, B), lam, r)
    with pytest.raises(AssertionError):
        ab.check("res", mut, res_ok, dres)
