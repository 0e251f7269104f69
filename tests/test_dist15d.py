"""Distributed FusedMM (Sec. V, c = 1) on CPU: the 1.5D dense-shifting
algorithm with local kernel fusion (Algorithm 1) and the 1.5D sparse-shifting
algorithm, 2 and 3 gloo ranks, local calls evaluated by the oracle, the
assembled outputs against the oracle on the whole matrix; and the index
arithmetic of the partitions."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2203_07673_gb300 import dist15d  # noqa: E402
from paper_2203_07673_gb300 import workloads as wl  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(world, seed, r, use_gpu, vals_none=False, body="rank_main", c=None, bf16=False):
    import dist15d_ranks
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = free_port()
    extra = () if c is None else (c,)
    if bf16:
        extra = (c or 1, True)
    procs = [ctx.Process(target=getattr(dist15d_ranks, body),
                         args=(k, world, port, out, seed, r, use_gpu, vals_none) + extra)
             for k in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return dict(out)


def assemble(res, world, S, r):
    """Every rank's output blocks into whole matrices; each row, column and
    nonzero must come from exactly one rank."""
    out = np.zeros((S.m, r)); out_t = np.zeros((S.n, r))
    dA = np.zeros((S.m, r)); dB = np.zeros((S.n, r)); ds = np.zeros(S.nnz)
    seen_r, seen_c, seen_nz = np.zeros(S.m, int), np.zeros(S.n, int), np.zeros(S.nnz, int)
    for k in range(world):
        r0, r1, c0, c1, slots = res[f"bounds{k}"]
        out[r0:r1] = res[k]["out"]; dA[r0:r1] = res[k]["dA"]; ds[slots] = res[k]["ds"]
        out_t[c0:c1] = res[k]["out_t"]; dB[c0:c1] = res[k]["dB"]
        seen_r[r0:r1] += 1; seen_c[c0:c1] += 1; seen_nz[slots] += 1
    assert np.all(seen_r == 1) and np.all(seen_c == 1) and np.all(seen_nz == 1)
    return out, out_t, dA, dB, ds


def expected(S, vals, A, B, G):
    rp, ci, n = S.row_ptr, S.col_idx, S.n
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ga, gb, gs = oracle.fusedmm_grad(rp, ci, vals, A64, B64, G.astype(np.float64), n)
    return (oracle.fusedmm(rp, ci, vals, A64, B64, n), oracle.fusedmm_t(rp, ci, vals, A64, B64, n),
            ga, gb, gs)


def rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


def test_row_bounds_balance_nonzeros_and_cover_every_row():
    rng = np.random.default_rng(0)
    S = wl.random_csr(1000, 300, rng, mean_deg=8, hubs=((5, 900),))
    for parts in (1, 2, 3, 7):
        b = dist15d.row_bounds_by_nnz(S.row_ptr, parts)
        assert b[0] == 0 and b[-1] == S.m and np.all(np.diff(b) >= 0)
        counts = np.diff(S.row_ptr.astype(np.int64)[b])
        assert counts.sum() == S.nnz
        # a block misses its share by less than one row's nonzeros
        assert np.all(np.abs(counts - S.nnz / parts) <= S.degrees().max() + 1)
    cb = dist15d.col_bounds_uniform(250, 3)
    assert list(cb) == [0, 83, 166, 250]


def test_split_by_column_blocks_is_a_partition():
    rng = np.random.default_rng(1)
    S = wl.random_csr(200, 97, rng, mean_deg=6, dup_frac=0.1, unsorted=True)
    rp = torch.from_numpy(S.row_ptr); ci = torch.from_numpy(S.col_idx)
    cb = dist15d.col_bounds_uniform(S.n, 4)
    blocks = dist15d.split_by_column_blocks(rp, ci, cb)
    seen = np.concatenate([b[2].numpy() for b in blocks])
    assert np.array_equal(np.sort(seen), np.arange(S.nnz))
    row_of = np.repeat(np.arange(S.m), S.degrees())
    for l, (brp, bci, sel) in enumerate(blocks):
        sel = sel.numpy()
        assert np.all((S.col_idx[sel] >= cb[l]) & (S.col_idx[sel] < cb[l + 1]))
        assert np.array_equal(bci.numpy(), S.col_idx[sel] - cb[l])
        # rows of the block's CSR are the rows the selected nonzeros sit in,
        # in the input order within each row
        brow = np.repeat(np.arange(S.m), np.diff(brp.numpy().astype(np.int64)))
        assert np.array_equal(brow, row_of[sel])
        assert np.all(np.diff(sel)[np.diff(brow) == 0] > 0)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("vals_none", [False, True])
def test_ring_schedule_matches_the_whole_matrix(world, vals_none):
    import dist15d_ranks
    seed, r = 11 + world, 8
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=False, vals_none=vals_none)
    got = assemble(res, world, S, r)
    want = expected(S, None if vals_none else vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert rel(x, y) <= 1e-6, name


@pytest.mark.parametrize("world,c", [(2, 2), (4, 2), (4, 4)])
def test_replicated_grid_matches_the_whole_matrix(world, c):
    """Algorithm 1 with replication factor c: A all-gathered along each fiber
    of c ranks, B shifted around layers of world / c ranks, the FusedMMA
    output and dA reduce-scattered along the fiber."""
    import dist15d_ranks
    seed, r = 5 + world + c, 8
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=False, c=c)
    got = assemble(res, world, S, r)
    want = expected(S, vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert rel(x, y) <= 1e-6, name


def test_replicated_grid_with_bf16_blocks():
    """BF16 A and B on a 2 x 2 grid: the all-gathered and shifted blocks
    travel as raw bytes; the result equals the oracle on the BF16-rounded
    inputs."""
    import dist15d_ranks
    world, c, seed, r = 4, 2, 19, 8
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=False, c=c, bf16=True)
    got = assemble(res, world, S, r)
    rnd = lambda X: torch.from_numpy(X).to(torch.bfloat16).float().numpy()  # noqa: E731
    want = expected(S, vals, rnd(A), rnd(B), G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert rel(x, y) <= 1e-6, name


@pytest.mark.parametrize("world,c", [(2, 1), (3, 1), (2, 2), (4, 2), (4, 4)])
@pytest.mark.parametrize("vals_none", [False, True])
def test_replication_reuse_matches_the_whole_matrix(world, c, vals_none):
    """FusedMMA by replication reuse: B all-gathered once along the fiber,
    an SDDMM round with A travelling, an SpMM round with the output
    travelling; no reduce-scatter."""
    import dist15d_ranks
    seed, r = 61 + 3 * world + c, 8
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=False, vals_none=vals_none, body="reuse_rank_main",
                    c=c)
    out = np.zeros((S.m, r))
    seen = np.zeros(S.m, int)
    for k in range(world):
        r0, r1 = res[f"bounds{k}"]
        out[r0:r1] = res[k]["out"]
        seen[r0:r1] += 1
    assert np.all(seen == 1)
    want = expected(S, None if vals_none else vals, A, B, G)[0]
    assert rel(out, want) <= 1e-6


def test_local_blocks_of_the_grid_partition_s():
    """The local S of every rank of a (p/c) x c grid, for both layouts,
    together hold every nonzero exactly once, with its row and column."""
    rng = np.random.default_rng(7)
    S = wl.random_csr(300, 170, rng, mean_deg=7, dup_frac=0.1, unsorted=True,
                      hubs=((4, 150),))
    rp, ci = torch.from_numpy(S.row_ptr), torch.from_numpy(S.col_idx)
    row_of = np.repeat(np.arange(S.m), S.degrees())
    for p, c in ((4, 2), (6, 3), (6, 2), (5, 1)):
        rb, cb = dist15d.row_bounds_by_nnz(S.row_ptr, p), dist15d.col_bounds_uniform(S.n, p)
        lp = p // c
        for layout in ("lkf", "reuse"):
            seen = np.zeros(S.nnz, int)
            for k in range(p):
                layer, q = divmod(k, lp)
                if layout == "lkf":
                    rr = (int(rb[q * c]), int(rb[(q + 1) * c]))
                    cc = (int(cb[layer * lp]), int(cb[(layer + 1) * lp]))
                else:
                    rr = (int(rb[layer * lp]), int(rb[(layer + 1) * lp]))
                    cc = (int(cb[q * c]), int(cb[(q + 1) * c]))
                lrp, lci, slots = dist15d.local_block(rp, ci, *rr, *cc)
                slots = slots.numpy()
                seen[slots] += 1
                assert np.array_equal(lci.numpy(), S.col_idx[slots])
                lrow = np.repeat(np.arange(rr[1] - rr[0]), np.diff(lrp.numpy().astype(np.int64)))
                assert np.array_equal(lrow + rr[0], row_of[slots])
                assert np.all((S.col_idx[slots] >= cc[0]) & (S.col_idx[slots] < cc[1]))
            assert np.all(seen == 1), (p, c, layout)


def test_one_rank_without_a_process_group():
    """p = 1 when no process group exists: one phase, no shift."""
    import dist15d_ranks
    S, vals, A, B, G = dist15d_ranks.problem(3, r=8)
    d = dist15d.FusedMM15D(torch.from_numpy(S.row_ptr), torch.from_numpy(S.col_idx), S.n, 8,
                           torch.float32, ops=dist15d_ranks.OracleOps())
    assert d.p == 1 and d.k == 0
    Vt, At, Bt, Gt = (torch.from_numpy(x) for x in (vals, A, B, G))
    got = (d.fusedmm(Vt, At, Bt), d.fusedmm_t(Vt, At, Bt)) + d.fusedmm_bwd(Vt, At, Bt, Gt)
    want = expected(S, vals, A, B, G)
    for x, y in zip(got, want):
        assert rel(x.double().numpy(), y) <= 1e-6


def assemble_slices(res, world, S, r):
    """Every rank's (rows, column slice) blocks into whole matrices; every
    element must come from exactly one rank."""
    out = np.zeros((S.m, r)); out_t = np.zeros((S.n, r))
    seen, seen_t = np.zeros((S.m, r), int), np.zeros((S.n, r), int)
    for k in range(world):
        j0, j1, r0, r1, c0, c1 = res[f"slice{k}"]
        out[r0:r1, j0:j1] = res[k]["out"]; out_t[c0:c1, j0:j1] = res[k]["out_t"]
        seen[r0:r1, j0:j1] += 1; seen_t[c0:c1, j0:j1] += 1
    assert np.all(seen == 1) and np.all(seen_t == 1)
    return out, out_t


@pytest.mark.parametrize("world,c", [(2, 1), (3, 1), (2, 2), (4, 2), (4, 4)])
@pytest.mark.parametrize("vals_none", [False, True])
def test_sparse_shifting_matches_the_whole_matrix(world, c, vals_none):
    """Sparse shifting on the (world/c) x c grid: block rows circulate in
    each layer, B is all-gathered along the fiber, FusedMMB reduce-scattered
    along it."""
    import dist15d_ranks
    seed, r = 31 + world + c, 9
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=False, vals_none=vals_none, body="sparse_rank_main",
                    c=c)
    got = assemble_slices(res, world, S, r)
    want = expected(S, None if vals_none else vals, A, B, G)[:2]
    for name, x, y in zip(("out", "out_t"), got, want):
        assert rel(x, y) <= 1e-6, name


def test_slice_bounds_cover_the_width():
    for r, parts in ((9, 2), (64, 3), (5, 5)):
        b = dist15d.slice_bounds(r, parts)
        assert b[0] == 0 and b[-1] == r and np.all(np.diff(b) >= 1)
