"""Pins of the oracle's graph-attention forward (Sec. VI-E) against closed
forms and a dense brute force written independently with numpy."""
import numpy as np
import pytest

import oracle
from paper_2203_07673_gb300 import workloads as wl


def _problem(seed, m=40, n=30, heads=2, rh=3, dup=0.0):
    rng = np.random.default_rng(seed)
    S = wl.random_csr(m, n, rng, mean_deg=4, empty_frac=0.2, dup_frac=dup)
    f = rng.standard_normal((m, heads))
    g = rng.standard_normal((n, heads))
    H = rng.standard_normal((n, heads * rh))
    vals = rng.uniform(0.5, 1.5, S.nnz)
    return S, vals, f, g, H


def _distinct_pattern(seed, m=40, n=30):
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 7, m)
    cols = [np.sort(rng.choice(n, d, replace=False)) for d in deg]
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    ci = np.concatenate(cols).astype(np.int32)
    return wl.CSR(m, n, rp, ci), rng


def test_dense_brute_force():
    S, rng = _distinct_pattern(1)
    heads = 2
    f = rng.standard_normal((S.m, heads)); g = rng.standard_normal((S.n, heads))
    H = rng.standard_normal((S.n, heads * 3)); vals = rng.uniform(0.5, 1.5, S.nnz)
    heads, rh, slope = 2, 3, 0.2
    got = oracle.gat(S.row_ptr, S.col_idx, vals, f, g, H, heads, slope)
    D = np.zeros((S.m, S.n)); mask = np.zeros((S.m, S.n), bool)
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
    D[rows, S.col_idx] = vals; mask[rows, S.col_idx] = True   # patterns without duplicates
    for h in range(heads):
        x = D * (f[:, h][:, None] + g[:, h][None, :])
        e = np.where(x > 0, x, slope * x)
        e = np.where(mask, e, -np.inf)
        with np.errstate(invalid="ignore"):
            a = np.exp(e - e.max(axis=1, keepdims=True))
            a = np.where(mask, a, 0.0)
            a = a / np.maximum(a.sum(axis=1, keepdims=True), 1e-300)
        exp = a @ H[:, h * rh:(h + 1) * rh]
        np.testing.assert_allclose(got[:, h * rh:(h + 1) * rh], exp, rtol=1e-12, atol=1e-12)


def test_uniform_scores_give_neighbour_means():
    S, vals, f, g, H = _problem(2, dup=0.3)
    got = oracle.gat(S.row_ptr, S.col_idx, None, np.zeros_like(f), np.zeros_like(g), H, 2, 0.2)
    for i in range(S.m):
        nb = S.col_idx[S.row_ptr[i]:S.row_ptr[i + 1]]
        exp = H[nb].mean(axis=0) if nb.size else np.zeros(H.shape[1])
        np.testing.assert_allclose(got[i], exp, rtol=1e-12, atol=1e-12)


def test_single_neighbour_and_shift_invariance():
    S, vals, f, g, H = _problem(3)
    rp = np.arange(S.m + 1); ci = np.arange(S.m) % S.n
    got = oracle.gat(rp, ci, None, f, g, H, 2, 0.2)
    np.testing.assert_allclose(got, H[ci], rtol=1e-12, atol=1e-12)
    # with all scores positive, adding c to f_i shifts every e_ij of row i by
    # c (times s = 1): the softmax, hence the output, is unchanged
    fpos, gpos = np.abs(f) + 1.0, np.abs(g) + 1.0
    a = oracle.gat(S.row_ptr, S.col_idx, None, fpos, gpos, H, 2, 0.2)
    b = oracle.gat(S.row_ptr, S.col_idx, None, fpos + 5.0, gpos, H, 2, 0.2)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_leaky_slope_matters_only_for_negative_scores():
    S, vals, f, g, H = _problem(4)
    fpos, gpos = np.abs(f) + 0.1, np.abs(g) + 0.1
    a = oracle.gat(S.row_ptr, S.col_idx, vals, fpos, gpos, H, 2, 0.2)
    b = oracle.gat(S.row_ptr, S.col_idx, vals, fpos, gpos, H, 2, 0.01)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    c = oracle.gat(S.row_ptr, S.col_idx, vals, -fpos, -gpos, H, 2, 0.01)
    assert not np.allclose(a, c)


def test_float32_inputs_match_float64_inputs():
    # the loader widens float32 arrays to float64 copies; those copies must
    # live through the call (float32 and float64 inputs give the same result)
    S, vals, f, g, H = _problem(6)
    a = oracle.gat(S.row_ptr, S.col_idx, vals, f, g, H, 2, 0.2)
    b = oracle.gat(S.row_ptr, S.col_idx, vals.astype(np.float32).astype(np.float64),
                   f.astype(np.float32), g.astype(np.float32), H.astype(np.float32), 2, 0.2)
    c = oracle.gat(S.row_ptr, S.col_idx, vals.astype(np.float32), f.astype(np.float32),
                   g.astype(np.float32), H.astype(np.float32), 2, 0.2)
    np.testing.assert_array_equal(b, c)
    np.testing.assert_allclose(a, c, rtol=1e-5, atol=1e-6)
