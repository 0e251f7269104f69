"""Element-wise error bounds of one float32 CG step of ALS (Sec. VI-E).

Both sides start a step from the same float32 state (x, res, p, rs), widened
exactly to float64 for the oracle, so the only differences are the float32
roundings of that one step.  Each bound is the first-order propagation of
those roundings through the step, computed per element from magnitudes the
oracle evaluates on absolute values; u = 2^-24, and the comparison allows a
factor 2 for the second-order terms.

Roundings counted (d = the row's nonzeros, r the width):
  SpMM  b = sum_j c_ij Y_j               |db|  <= 2 (d + 2) u  Bm,  Bm = SpMM(|c|, |Y|)
  FusedMM q = sum_j <x, Y_j> Y_j          |dq|  <= 2 (r + d + 4) u Q,   Q = FusedMM(|x|, |Y|)
  init  res = b - q - lam x               |dres| <= |db| + |dq| + 3u (|b| + |q| + lam |x|)
  step  t = q + lam p                     |dt|  <= |dq| + 2u T,  T = Q + lam |p|
        pt = <p, t>                       |dpt| <= sum |p| |dt| + (r + 1) u sum |p| T
        alpha = rs / pt                   |da|  <= |alpha| (|dpt| / |pt| + u)
        x' = x + alpha p                  |dx'| <= |da| |p| + 2u (|x| + |alpha p|)
        res' = res - alpha t              |dres'| <= |da| |t| + |alpha| |dt| + 2u (|res| + |alpha t|)
        rs' = <res', res'>                |drs'| <= 2 sum |res'| |dres'| + (r + 1) u sum res'^2
        beta = rs' / rs                   |db'| <= |drs'| / rs + u |beta|
        p' = res' + beta p                |dp'| <= |dres'| + |db'| |p| + 2u (|res'| + |beta p|)
The pt term is evaluated with the step's own numbers, so it carries the
conditioning of the row's system (sum |p| T / <p, t> is at most about the
condition number of M_i) without assuming a value for it.
"""
import numpy as np

import oracle

U32 = 2.0 ** -24
SLACK = 2.0


def side_degrees(S, side):
    if side == 0:
        return np.diff(S.row_ptr.astype(np.int64))
    return np.bincount(S.col_idx, minlength=S.n).astype(np.int64)


def _fusedmm(S, side, X, Y):
    """M' X (the FusedMM of the 0/1 pattern, without lambda) of the side."""
    rp, ci, n = S.row_ptr, S.col_idx, S.n
    if side == 0:
        return oracle.fusedmm(rp, ci, None, X, Y, n)
    return oracle.fusedmm_t(rp, ci, None, Y, X, n)


def _spmm(S, side, c, Y):
    rp, ci, n = S.row_ptr, S.col_idx, S.n
    if side == 0:
        return oracle.spmm(rp, ci, c, Y, n)
    return oracle.spmm_t(rp, ci, c, Y, n)


def init_bound(S, side, c, X, Y, lam, r):
    """Bounds of (res, rs) after the set-up from X (the side being updated)
    with Y the fixed factor; p = res exactly."""
    d = side_degrees(S, side)[:, None].astype(np.float64)
    b = _spmm(S, side, c, Y)
    q = _fusedmm(S, side, X, Y)
    Bm = _spmm(S, side, np.abs(c), np.abs(Y))
    Q = _fusedmm(S, side, np.abs(X), np.abs(Y))
    db = 2 * (d + 2) * U32 * Bm
    dq = 2 * (r + d + 4) * U32 * Q
    res = b - q - lam * X
    dres = db + dq + 3 * U32 * (np.abs(b) + np.abs(q) + lam * np.abs(X))
    drs = 2 * (np.abs(res) * dres).sum(1) + (r + 1) * U32 * (res * res).sum(1)
    return dres, drs


def step_bound(S, side, X, res, p, rs, Y, lam, r):
    """Bounds of (x', res', p', rs') after one CG step from the state
    (X, res, p, rs) with Y fixed."""
    d = side_degrees(S, side)[:, None].astype(np.float64)
    q = _fusedmm(S, side, p, Y)
    Q = _fusedmm(S, side, np.abs(p), np.abs(Y))
    t = q + lam * p
    T = Q + lam * np.abs(p)
    dt = 2 * (r + d + 4) * U32 * Q + 2 * U32 * T
    pt = (p * t).sum(1)
    dpt = (np.abs(p) * dt).sum(1) + (r + 1) * U32 * (np.abs(p) * T).sum(1)
    pos = pt > 0
    alpha = np.where(pos, rs / np.where(pos, pt, 1.0), 0.0)
    da = np.where(pos, np.abs(alpha) * (dpt / np.abs(np.where(pos, pt, 1.0)) + U32), 0.0)
    a, da = alpha[:, None], da[:, None]
    x1 = X + a * p
    res1 = res - a * t
    dx = da * np.abs(p) + 2 * U32 * (np.abs(X) + np.abs(a * p))
    dres = da * np.abs(t) + np.abs(a) * dt + 2 * U32 * (np.abs(res) + np.abs(a * t))
    rs1 = (res1 * res1).sum(1)
    drs = 2 * (np.abs(res1) * dres).sum(1) + (r + 1) * U32 * rs1
    posr = rs > 0
    beta = np.where(posr, rs1 / np.where(posr, rs, 1.0), 0.0)
    dbeta = np.where(posr, drs / np.where(posr, rs, 1.0) + U32 * np.abs(beta), 0.0)
    dp = dres + dbeta[:, None] * np.abs(p) + 2 * U32 * (np.abs(res1) + np.abs(beta[:, None] * p))
    return dx, dres, dp, drs


def check(name, got, ref, bound):
    """Every element within SLACK x its bound; returns the largest ratio."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), name
    lim = SLACK * bound + 1e-300
    err = np.abs(got - ref)
    bad = err > lim
    if bad.any():
        idx = tuple(np.argwhere(bad)[0])
        raise AssertionError(f"{name}: {int(bad.sum())} elements over the bound; first at {idx}: "
                             f"got={got[idx]!r} oracle={ref[idx]!r} bound={lim[idx]!r}")
    return float((err / lim).max()) if err.size else 0.0


def row_condition(S, side, Y, lam):
    """Condition number of every row's M_i = sum_j Y_j Y_j^T + lam I."""
    rp = S.row_ptr.astype(np.int64)
    r = Y.shape[1]
    if side == 0:
        nbrs = [S.col_idx[rp[i]:rp[i + 1]] for i in range(S.m)]
    else:
        rows_of = np.repeat(np.arange(S.m), np.diff(rp))
        order = np.argsort(S.col_idx, kind="stable")
        starts = np.searchsorted(S.col_idx[order], np.arange(S.n + 1))
        nbrs = [rows_of[order[starts[j]:starts[j + 1]]] for j in range(S.n)]
    kappa = np.empty(len(nbrs))
    for i, nb in enumerate(nbrs):
        Yn = Y[nb]
        ev = np.linalg.eigvalsh(Yn.T @ Yn + lam * np.eye(r))
        kappa[i] = ev[-1] / ev[0]
    return kappa
