"""Shared helpers of the GPU parity tests: upload inputs, run the oracle, and
compare element by element.

Tolerances.  The stated bar is a relative Frobenius error <= 1e-5 for float32
inputs and <= 2e-2 for bfloat16 inputs against the FP64 oracle fed the
original float32 samples.  On top of it every element must satisfy the
float32 rounding bound of its own sum:

    |x_gpu - x_oracle| <= 2 * (r + deg_max + 4) * 2^-24 * M

where M is the same result computed by the oracle on |s|, |A|, |B| (and |G|):
the sum of the magnitudes of every product that enters the element.  A dot
product of r terms, one scaling and an accumulation of deg terms each add at
most (terms) * u relative to that magnitude sum (u = 2^-24); the factor 2 is
slack.  For bfloat16 runs the oracle is fed the bfloat16-rounded inputs
(widened exactly), so the same bound applies, and the error against the
original float32 samples is reported separately.
"""
import numpy as np
import torch

import oracle

U32 = 2.0 ** -24


def upload(S, vals, A, B, dtype=torch.float32, device="cuda"):
    rp = torch.from_numpy(np.ascontiguousarray(S.row_ptr)).to(device)
    ci = torch.from_numpy(np.ascontiguousarray(S.col_idx)).to(device)
    v = None if vals is None else torch.from_numpy(np.ascontiguousarray(vals, np.float32)).to(device)
    At = torch.from_numpy(np.ascontiguousarray(A, np.float32)).to(device).to(dtype).contiguous()
    Bt = torch.from_numpy(np.ascontiguousarray(B, np.float32)).to(device).to(dtype).contiguous()
    return rp, ci, v, At, Bt


def host64(t):
    """Exactly the values the GPU received, widened to float64."""
    return None if t is None else t.detach().cpu().double().numpy()


def relF(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(x - ref)
    return 0.0 if num == 0 else num / max(den, 1e-300)


def assert_close(name, gpu, ref, mag, r, deg_max, rel_tol=1e-5):
    gpu = gpu.detach().cpu().double().numpy() if isinstance(gpu, torch.Tensor) else gpu
    assert gpu.shape == ref.shape, (name, gpu.shape, ref.shape)
    assert np.all(np.isfinite(gpu)), name
    bound = 2.0 * (r + deg_max + 4) * U32 * mag + 1e-30
    err = np.abs(gpu - ref)
    bad = err > bound
    if bad.any():
        idx = np.argwhere(bad)[0]
        raise AssertionError(f"{name}: {bad.sum()} elements over the rounding bound; first at "
                             f"{tuple(idx)}: gpu={gpu[tuple(idx)]!r} oracle={ref[tuple(idx)]!r} "
                             f"bound={bound[tuple(idx)]!r}")
    e = relF(gpu, ref)
    assert e <= rel_tol, f"{name}: relative Frobenius error {e:.3e} > {rel_tol:g}"
    return e


def deg_max(S):
    rows = int(S.degrees().max()) if S.m else 0
    cols = int(np.bincount(S.col_idx, minlength=max(S.n, 1)).max()) if S.nnz else 0
    return max(rows, cols)


def oracle_all(S, vals, A, B, G, Gn):
    """Every result of the library, by the oracle, in float64."""
    rp, ci, n = S.row_ptr, S.col_idx, S.n
    res = dict(
        fusedmm=oracle.fusedmm(rp, ci, vals, A, B, n),
        fusedmm_t=oracle.fusedmm_t(rp, ci, vals, A, B, n),
        sddmm=oracle.sddmm(rp, ci, vals, A, B, n),
    )
    v = res["sddmm"]
    res["spmm"] = oracle.spmm(rp, ci, v, B, n)
    res["spmm_t"] = oracle.spmm_t(rp, ci, v, A, n)
    res["bwd"] = oracle.fusedmm_grad(rp, ci, vals, A, B, G, n)
    res["t_bwd"] = oracle.fusedmm_t_grad(rp, ci, vals, A, B, Gn, n)
    return res


def absolute(x):
    return None if x is None else np.abs(x)


def rows_problem(S, rows, vals=None):
    """The sub-pattern of the given rows (in the given order) with its
    columns compacted: returns (row_ptr, col_idx, vals, cols, nnz_index) so
    that FusedMMA of the sub-problem on (A[rows], B[cols]) gives exactly
    those rows of the full result."""
    rp = S.row_ptr.astype(np.int64)
    deg = rp[rows + 1] - rp[rows]
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows]) if len(rows) else \
        np.zeros(0, np.int64)
    sub_rp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(deg, out=sub_rp[1:])
    cols, ci = np.unique(S.col_idx[idx], return_inverse=True)
    v = None if vals is None else np.asarray(vals)[idx]
    return sub_rp, ci.astype(np.int64), v, cols, idx


def cols_problem(S, cols, vals=None):
    """The nonzeros of S in the given columns: returns (row_ptr, col_idx,
    vals, rows, nnz_index) with rows compacted and column c of the
    sub-problem being cols[c], so that FusedMMB of the sub-problem on
    (A[rows], B[cols]) gives exactly those columns of the full result."""
    cols = np.asarray(cols)
    pos = np.full(S.n, -1, np.int64)
    pos[cols] = np.arange(len(cols))
    sel = pos[S.col_idx] >= 0
    idx = np.nonzero(sel)[0]
    row_of = np.repeat(np.arange(S.m), np.diff(S.row_ptr.astype(np.int64)))
    r_sel = row_of[idx]
    rows, r_new = np.unique(r_sel, return_inverse=True)
    sub_rp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(np.bincount(r_new, minlength=len(rows)), out=sub_rp[1:])
    v = None if vals is None else np.asarray(vals)[idx]
    return sub_rp, pos[S.col_idx[idx]], v, rows, idx
