"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out: CSR patterns (row
pointers and column indices, int32), values of S and dense row-major
matrices.  It holds none of the FusedMM arithmetic, and it is the one module
that both the CUDA path and the FP64 oracle are fed from: a test draws its
inputs here and hands the same arrays to each side.

Patterns:
  * ``er_exact_degree``  Erdos-Renyi with exactly ``deg`` distinct uniform
    columns per row (the paper's weak-scaling matrices, Sec. VI-B, 32 nonzeros
    per row).
  * ``rmat``             R-MAT power-law graph with a random vertex relabeling
    (a stand-in for the SuiteSparse graphs of Sec. VI-D, which are not used;
    the relabeling mirrors the random row/column permutation of Sec. VI).
  * ``zipf_rows``        rectangular S with Zipf-distributed row degrees and
    uniform distinct columns (the ALS-shaped workload of Sec. VI-E).
  * ``random_csr``       small irregular patterns for tests: empty rows,
    unsorted or duplicate columns, hub rows.

Every workload takes a ``numpy.random.Generator``; ``config_rng(k, stream)``
gives the seeded generator of array ``stream`` of workload ``k``
(PCG64, root seed 2203_07673 + k).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ROOT_SEED = 220307673


def config_rng(config_index: int, stream: int) -> np.random.Generator:
    """Independent PCG64 stream ``stream`` of workload ``config_index``."""
    ss = np.random.SeedSequence([ROOT_SEED + int(config_index), int(stream)])
    return np.random.Generator(np.random.PCG64(ss))


@dataclasses.dataclass
class CSR:
    """CSR pattern with int32 indices (row_ptr has m + 1 entries)."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def rows_slice(self, r0: int, r1: int) -> "CSR":
        """Rows [r0, r1) as a CSR of their own (columns unchanged)."""
        base = int(self.row_ptr[r0])
        rp = (self.row_ptr[r0:r1 + 1].astype(np.int64) - base).astype(np.int32)
        ci = self.col_idx[base:int(self.row_ptr[r1])]
        return CSR(r1 - r0, self.n, rp, ci)


def _csr_from_sorted_keys(keys: np.ndarray, m: int, n: int) -> CSR:
    rows = (keys // n).astype(np.int64)
    cols = (keys % n).astype(np.int32)
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("pattern has 2^31 or more nonzeros")
    return CSR(m, n, row_ptr.astype(np.int32), cols)


def _distinct_columns(rows: np.ndarray, m: int, n: int,
                      rng: np.random.Generator) -> CSR:
    """Uniform columns for the given row of every nonzero, redrawn until the
    columns of each row are distinct; returned sorted within each row."""
    rows = rows.astype(np.int64)
    cols = rng.integers(0, n, size=rows.shape[0], dtype=np.int64)
    while True:
        keys = rows * n + cols
        order = np.argsort(keys, kind="stable")
        keys = keys[order]
        rows = rows[order]
        dup = np.zeros(keys.shape[0], bool)
        if keys.shape[0] > 1:
            dup[1:] = keys[1:] == keys[:-1]
        nd = int(dup.sum())
        cols = keys % n
        if nd == 0:
            return _csr_from_sorted_keys(keys, m, n)
        cols[dup] = rng.integers(0, n, size=nd, dtype=np.int64)


def er_exact_degree(m: int, n: int, deg: int, rng: np.random.Generator) -> CSR:
    """Erdos-Renyi pattern: exactly ``deg`` distinct uniform columns per row,
    sorted within the row."""
    if deg > n:
        raise ValueError("deg > n")
    if m == 0 or deg == 0:
        return CSR(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32))
    if deg * 4 > n:
        # dense-ish rows: a random subset per row from a per-row permutation
        cols = np.argsort(rng.random((m, n)), axis=1)[:, :deg]
        cols.sort(axis=1)
        row_ptr = (np.arange(m + 1, dtype=np.int64) * deg).astype(np.int32)
        return CSR(m, n, row_ptr, cols.reshape(-1).astype(np.int32))
    cols = rng.integers(0, n, size=(m, deg), dtype=np.int32)
    while True:
        cols.sort(axis=1)
        bad = np.nonzero((cols[:, 1:] == cols[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        cols[bad] = rng.integers(0, n, size=(bad.size, deg), dtype=np.int32)
    row_ptr = (np.arange(m + 1, dtype=np.int64) * deg).astype(np.int32)
    return CSR(m, n, row_ptr, cols.reshape(-1))


def rmat(scale: int, edge_factor: float, a: float, b: float, c: float,
         d: float, rng: np.random.Generator, vertices: int | None = None) -> CSR:
    """R-MAT graph on 2^scale vertices with edge_factor * 2^scale edge draws.

    Each draw picks one of the four quadrants per level with probabilities
    (a, b, c, d) for (row bit, col bit) = (0,0), (0,1), (1,0), (1,1).  The
    vertex ids are then relabeled by one random permutation (applied to rows
    and columns alike), duplicate (i, j) pairs are merged and self-loops are
    kept.  With ``vertices`` < 2^scale, ids are folded onto [0, vertices) by
    taking them modulo ``vertices`` after the relabeling.
    """
    assert abs(a + b + c + d - 1.0) < 1e-9
    nv = 1 << scale
    E = int(round(edge_factor * nv))
    rows = np.zeros(E, np.uint32)
    cols = np.zeros(E, np.uint32)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = rng.random(E, dtype=np.float32)
        rbit = u >= ab
        cbit = ((u >= a) & (u < ab)) | (u >= abc)
        bit = np.uint32(1 << (scale - 1 - level))
        rows |= rbit.astype(np.uint32) * bit
        cols |= cbit.astype(np.uint32) * bit
        del u, rbit, cbit
    perm = rng.permutation(nv).astype(np.uint32)
    rows = perm[rows]
    cols = perm[cols]
    V = nv if vertices is None else int(vertices)
    if V != nv:
        rows %= np.uint32(V)
        cols %= np.uint32(V)
    keys = rows.astype(np.int64) * V + cols.astype(np.int64)
    del rows, cols
    keys = np.unique(keys)
    return _csr_from_sorted_keys(keys, V, V)


def zipf_degrees(m: int, total_nnz: int, alpha: float, dmax: int,
                 rng: np.random.Generator, n: int | None = None) -> np.ndarray:
    """Row degrees d_i = clip(round(c * w_i), 1, dmax) with w_i drawn from
    Zipf(alpha) truncated to [1, dmax] and c found by bisection so that
    sum(d_i) is within 0.1% of total_nnz (np.round: ties to even)."""
    k = np.arange(1, dmax + 1, dtype=np.float64)
    pmf = k ** (-alpha)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    w = (np.searchsorted(cdf, rng.random(m), side="right") + 1).astype(np.float64)
    w = np.minimum(w, dmax)
    cap = dmax if n is None else min(dmax, n)

    def degs(c):
        return np.clip(np.round(c * w), 1, cap).astype(np.int64)

    lo, hi = 0.0, float(cap)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = int(degs(mid).sum())
        if abs(s - total_nnz) <= 0.001 * total_nnz:
            return degs(mid)
        if s < total_nnz:
            lo = mid
        else:
            hi = mid
    return degs(0.5 * (lo + hi))


def zipf_rows(m: int, n: int, total_nnz: int, alpha: float, dmax: int,
              rng: np.random.Generator) -> CSR:
    """Rectangular m x n pattern with Zipf row degrees (``zipf_degrees``) and
    uniform distinct columns within each row, sorted within the row."""
    d = zipf_degrees(m, total_nnz, alpha, dmax, rng, n=n)
    rows = np.repeat(np.arange(m, dtype=np.int64), d)
    return _distinct_columns(rows, m, n, rng)


def random_csr(m: int, n: int, rng: np.random.Generator, mean_deg: float = 4.0,
               empty_frac: float = 0.2, dup_frac: float = 0.0,
               unsorted: bool = False, hubs: tuple = ()) -> CSR:
    """Irregular small pattern for tests.

    Row degrees are Poisson(mean_deg); a fraction ``empty_frac`` of the rows is
    forced empty; ``hubs`` lists (row, degree) pairs of long rows.  Columns are
    uniform; a fraction ``dup_frac`` of the nonzeros repeats the previous
    column of the same row, and with ``unsorted`` each row's columns are
    shuffled, otherwise sorted.
    """
    deg = rng.poisson(mean_deg, size=m).astype(np.int64)
    if m:
        deg[rng.random(m) < empty_frac] = 0
    for row, dg in hubs:
        deg[row] = dg
    if n == 0:
        deg[:] = 0
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    cols = rng.integers(0, max(n, 1), size=nnz, dtype=np.int64)
    for i in range(m):
        a, b = row_ptr[i], row_ptr[i + 1]
        if b - a == 0:
            continue
        seg = cols[a:b]
        if not unsorted:
            seg.sort()
        if dup_frac > 0 and b - a > 1:
            rep = np.nonzero(rng.random(b - a - 1) < dup_frac)[0] + 1
            for t in rep:
                seg[t] = seg[t - 1]
        if unsorted:
            rng.shuffle(seg)
    return CSR(m, n, row_ptr.astype(np.int32), cols.astype(np.int32))


def normal(rows: int, r: int, variance: float, rng: np.random.Generator) -> np.ndarray:
    """rows x r float32 matrix with entries N(0, variance)."""
    x = rng.standard_normal((rows, r), dtype=np.float32)
    x *= np.float32(math.sqrt(variance))
    return x


def uniform(count: int, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(lo, hi, size=count).astype(np.float32)


def half_steps(count: int, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    """U(lo, hi) rounded to the nearest multiple of 0.5 (ties to even)."""
    return (np.round(rng.uniform(lo, hi, size=count) * 2.0) / 2.0).astype(np.float32)


def small_ints(shape, bound: int, rng: np.random.Generator) -> np.ndarray:
    """Integers in [-bound, bound] as float32 (exact-arithmetic test inputs)."""
    return rng.integers(-bound, bound + 1, size=shape).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads.  Each returns a dict with the pattern ``S`` (CSR),
# ``vals`` (float32 or None for s == 1), ``A``, ``B`` (float32), ``r``, the
# input dtype name and a description.  ``scale_rows`` shrinks the row count
# of the large ones for quick checks (1.0 = the full workload).

WORKLOADS = {
    1: "ER 4096x4096, 32 nnz/row, r=32, FP32, s~U(0,1), A,B~N(0,1)",
    2: "ER 2^20x2^20, 32 nnz/row, r=128, FP32, s~U(0,1), A,B~N(0,1/128)",
    3: "R-MAT 2^22 (a,b,c,d)=(.57,.19,.19,.05), avg deg 16, s=1, r=64, BF16, A,B~N(0,1/64)",
    4: "Zipf(1.2) rows 2^21x2^19, 80M nnz, r=64, s in {1,1.5,..,5}, A,B~N(0,0.1)",
    5: "512 uneven matrices (ER 8-64/row, R-MAT deg 16), r in {32,64,128}, BF16",
}


def workload(k: int, scale_rows: float = 1.0) -> dict:
    if k == 1:
        m = n = max(1, int(4096 * scale_rows))
        S = er_exact_degree(m, n, min(32, n), config_rng(1, 0))
        return dict(S=S, vals=uniform(S.nnz, 0.0, 1.0, config_rng(1, 1)),
                    A=normal(m, 32, 1.0, config_rng(1, 2)),
                    B=normal(n, 32, 1.0, config_rng(1, 3)),
                    r=32, dtype="f32", name=WORKLOADS[1])
    if k == 2:
        m = n = max(1, int((1 << 20) * scale_rows))
        S = er_exact_degree(m, n, min(32, n), config_rng(2, 0))
        return dict(S=S, vals=uniform(S.nnz, 0.0, 1.0, config_rng(2, 1)),
                    A=normal(m, 128, 1.0 / 128, config_rng(2, 2)),
                    B=normal(n, 128, 1.0 / 128, config_rng(2, 3)),
                    r=128, dtype="f32", name=WORKLOADS[2])
    if k == 3:
        scale = 22
        while scale > 4 and (1 << scale) > (1 << 22) * scale_rows:
            scale -= 1
        S = rmat(scale, 16, 0.57, 0.19, 0.19, 0.05, config_rng(3, 0))
        nv = 1 << scale
        return dict(S=S, vals=None,
                    A=normal(nv, 64, 1.0 / 64, config_rng(3, 2)),
                    B=normal(nv, 64, 1.0 / 64, config_rng(3, 3)),
                    r=64, dtype="bf16", name=WORKLOADS[3])
    if k == 4:
        m = max(1, int((1 << 21) * scale_rows))
        n = max(1, int((1 << 19) * scale_rows))
        total = max(m, int(80_000_000 * scale_rows))
        S = zipf_rows(m, n, total, 1.2, 4096, config_rng(4, 0))
        return dict(S=S, vals=half_steps(S.nnz, 1.0, 5.0, config_rng(4, 1)),
                    A=normal(m, 64, 0.1, config_rng(4, 2)),
                    B=normal(n, 64, 0.1, config_rng(4, 3)),
                    r=64, dtype="f32", name=WORKLOADS[4])
    raise ValueError(f"unknown workload {k}")


def batched_specs(count: int = 512, seed_index: int = 5, rows_lo: float = 1e3,
                  rows_hi: float = 2e5, scale_rows: float = 1.0) -> list:
    """Per-matrix specs of the batched workload: rows log-uniform in
    [rows_lo, rows_hi] (times ``scale_rows``), even index Erdos-Renyi with a
    uniform degree in [8, 64], odd index R-MAT with average degree 16, and r
    uniform over {32, 64, 128}."""
    rng = config_rng(seed_index, 0)
    specs = []
    for t in range(count):
        rows = int(round(math.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi)))))
        rows = max(8, int(rows * scale_rows))
        r = int(rng.choice([32, 64, 128]))
        if t % 2 == 0:
            specs.append(dict(kind="er", rows=rows, deg=int(rng.integers(8, 65)), r=r))
        else:
            specs.append(dict(kind="rmat", rows=rows, deg=16, r=r))
    return specs


def batched_matrix(spec: dict, t: int, seed_index: int = 5) -> dict:
    """Materialise matrix ``t`` of the batched workload (BF16 inputs are the
    float32 samples rounded to bfloat16 by the caller)."""
    rng = config_rng(seed_index, 1000 + t)
    rows, r = spec["rows"], spec["r"]
    if spec["kind"] == "er":
        S = er_exact_degree(rows, rows, min(spec["deg"], rows), rng)
    else:
        scale = max(1, int(math.ceil(math.log2(rows))))
        S = rmat(scale, spec["deg"] * rows / (1 << scale), 0.57, 0.19, 0.19,
                 0.05, rng, vertices=rows)
    return dict(S=S, vals=uniform(S.nnz, 0.0, 1.0, rng),
                A=normal(rows, r, 1.0 / r, rng), B=normal(rows, r, 1.0 / r, rng),
                r=r)


# ---------------------------------------------------------------------------
# The batched workload drawn with torch on a device (same recipe as
# batched_matrix, a different random stream): 512 matrices are generated in
# seconds instead of minutes.  Returns device tensors; the oracle receives
# host copies of exactly these tensors.

def _torch_gen(device, seed):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def er_exact_degree_torch(m, n, deg, g, device):
    import torch
    deg = min(deg, n)
    cols = torch.randint(0, n, (m, deg), generator=g, device=device, dtype=torch.int64)
    while True:
        cols, _ = torch.sort(cols, dim=1)
        bad = (cols[:, 1:] == cols[:, :-1]).any(dim=1).nonzero().flatten() if deg > 1 else \
            torch.zeros(0, dtype=torch.int64, device=device)
        if bad.numel() == 0:
            break
        cols[bad] = torch.randint(0, n, (bad.numel(), deg), generator=g, device=device,
                                  dtype=torch.int64)
    row_ptr = torch.arange(m + 1, device=device, dtype=torch.int64) * deg
    return row_ptr.int(), cols.reshape(-1).int()


def rmat_torch(scale, edges, a, b, c, g, device, vertices):
    import torch
    E = int(edges)
    rows = torch.zeros(E, dtype=torch.int64, device=device)
    cols = torch.zeros(E, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = torch.rand(E, generator=g, device=device)
        bit = 1 << (scale - 1 - level)
        rows |= (u >= ab).long() * bit
        cols |= (((u >= a) & (u < ab)) | (u >= abc)).long() * bit
    perm = torch.randperm(1 << scale, generator=g, device=device)
    rows = perm[rows] % vertices
    cols = perm[cols] % vertices
    keys = torch.unique(rows * vertices + cols)
    r_, c_ = keys // vertices, keys % vertices
    counts = torch.bincount(r_, minlength=vertices)
    row_ptr = torch.zeros(vertices + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr.int(), c_.int()


def batched_matrix_torch(spec: dict, t: int, device, seed_index: int = 5) -> dict:
    """Matrix t of the batched workload as device tensors: row_ptr, col_idx
    (int32), vals ~ U(0,1), A, B ~ N(0, 1/r) (float32), r, m, n."""
    import torch
    g = _torch_gen(device, (ROOT_SEED + seed_index) * 1000003 + t)
    rows, r = spec["rows"], spec["r"]
    if spec["kind"] == "er":
        rp, ci = er_exact_degree_torch(rows, rows, spec["deg"], g, device)
    else:
        scale = max(1, int(math.ceil(math.log2(rows))))
        rp, ci = rmat_torch(scale, spec["deg"] * rows, 0.57, 0.19, 0.19, g, device, rows)
    nnz = ci.numel()
    vals = torch.rand(nnz, generator=g, device=device)
    std = math.sqrt(1.0 / r)
    A = torch.randn(rows, r, generator=g, device=device) * std
    B = torch.randn(rows, r, generator=g, device=device) * std
    return dict(row_ptr=rp, col_idx=ci, vals=vals, A=A, B=B, r=r, m=rows, n=rows)


# ---------------------------------------------------------------------------
# The Zipf-row workload (workload 4's recipe) drawn with torch on a device:
# the 80M-nonzero pattern in seconds instead of a minute on the host.  Same
# recipe as zipf_rows / workload(4), another random stream.

def zipf_degrees_torch(m, total_nnz, alpha, dmax, g, device, n=None):
    """Row degrees clip(round(c * w_i), 1, min(dmax, n)), w_i ~ Zipf(alpha)
    truncated to [1, dmax], c by bisection so that the sum is within 0.1 %
    of total_nnz (torch.round: ties to even, as np.round)."""
    import torch
    k = torch.arange(1, dmax + 1, dtype=torch.float64, device=device)
    cdf = torch.cumsum(k ** (-alpha), 0)
    cdf /= cdf[-1].clone()
    u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
    w = torch.clamp(torch.searchsorted(cdf, u, right=True) + 1, max=dmax).double()
    cap = dmax if n is None else min(dmax, n)

    def degs(c):
        return torch.clamp(torch.round(c * w), 1, cap).long()

    lo, hi = 0.0, float(cap)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = int(degs(mid).sum())
        if abs(s - total_nnz) <= 0.001 * total_nnz:
            return degs(mid)
        if s < total_nnz:
            lo = mid
        else:
            hi = mid
    return degs(0.5 * (lo + hi))


def zipf_rows_torch(m, n, total_nnz, alpha, dmax, g, device):
    """Device (row_ptr, col_idx) int32 of an m x n pattern with Zipf row
    degrees and uniform distinct columns, sorted within each row."""
    import torch
    d = zipf_degrees_torch(m, total_nnz, alpha, dmax, g, device, n=n)
    rows = torch.repeat_interleave(torch.arange(m, device=device, dtype=torch.int64), d)
    cols = torch.randint(0, n, rows.shape, generator=g, device=device, dtype=torch.int64)
    while True:
        keys, order = torch.sort(rows * n + cols)
        rows = rows[order]
        dup = torch.zeros_like(keys, dtype=torch.bool)
        if keys.numel() > 1:
            dup[1:] = keys[1:] == keys[:-1]
        nd = int(dup.sum())
        cols = keys % n
        if nd == 0:
            break
        cols[dup] = torch.randint(0, n, (nd,), generator=g, device=device, dtype=torch.int64)
    del keys, order, dup
    counts = torch.bincount(rows, minlength=m)
    row_ptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr.int(), cols.int()


def zipf_workload_torch(device, scale_rows: float = 1.0, seed_index: int = 4) -> dict:
    """Workload 4 as device tensors: 2^21 x 2^19 (times scale_rows) Zipf(1.2)
    rows in [1, 4096] with 80M nonzeros, s in {1, 1.5, ..., 5}, A, B ~
    N(0, 0.1) float32, r = 64."""
    import torch
    g = _torch_gen(device, (ROOT_SEED + seed_index) * 1000003 + 77)
    m = max(1, int((1 << 21) * scale_rows))
    n = max(1, int((1 << 19) * scale_rows))
    total = max(m, int(80_000_000 * scale_rows))
    rp, ci = zipf_rows_torch(m, n, total, 1.2, 4096, g, device)
    nnz = ci.numel()
    vals = torch.round((torch.rand(nnz, generator=g, device=device) * 4.0 + 1.0) * 2.0) / 2.0
    std = math.sqrt(0.1)
    A = torch.randn(m, 64, generator=g, device=device) * std
    B = torch.randn(n, 64, generator=g, device=device) * std
    return dict(row_ptr=rp, col_idx=ci, vals=vals, A=A, B=B, r=64, m=m, n=n,
                name=WORKLOADS[4] + " [drawn on the device]")
