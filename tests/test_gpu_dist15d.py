"""1.5D dense-shifting FusedMM with local kernel fusion (Sec. V, Algorithm 1,
c = 1) with the library's kernels: two gloo ranks on the one GPU (the
shifts staged through host memory; no kernel waits on another rank), the
assembled FusedMMA, FusedMMB, dA, dB and ds against the FP64 oracle on the
whole matrix, within the float32 parity bar.  Each local call covers one
column block of the rank's rows: phase 0 writes the outputs (fmm_fusedmm,
fmm_fusedmm_t, fmm_fusedmm_bwd), later phases add to them (fmm_fusedmm_acc,
fmm_fusedmm_t_acc, fmm_fusedmm_bwd_acc)."""
import numpy as np
import pytest

from test_dist15d import assemble, assemble_slices, expected, rel, run_ranks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r", [32, 24])
@pytest.mark.parametrize("vals_none", [False, True])
def test_two_ranks_on_one_gpu_match_the_whole_matrix(r, vals_none):
    import dist15d_ranks
    seed = 21 + r
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(2, seed, r, use_gpu=True, vals_none=vals_none)
    got = assemble(res, 2, S, r)
    want = expected(S, None if vals_none else vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


def test_three_ranks_with_a_padded_block():
    """n = 250 over 3 ranks: blocks of 83, 83 and 84 columns, so two ranks
    pad their B block to the 84 rows every shift moves."""
    import dist15d_ranks
    seed, r = 51, 32
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(3, seed, r, use_gpu=True)
    got = assemble(res, 3, S, r)
    want = expected(S, vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


def test_one_rank_without_a_process_group_on_the_gpu():
    """p = 1: one phase of write-mode calls, B and the values used in place."""
    import torch
    import dist15d_ranks
    from paper_2203_07673_gb300 import dist15d
    S, vals, A, B, G = dist15d_ranks.problem(61, r=64)
    dev = torch.device("cuda", 0)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    d = dist15d.FusedMM15D(t(S.row_ptr), t(S.col_idx), S.n, 64, torch.float32)
    assert d.p == 1 and d.spans == [(0, S.nnz)]
    V, A_d, B_d, G_d = t(vals), t(A), t(B), t(G)
    got = (d.fusedmm(V, A_d, B_d), d.fusedmm_t(V, A_d, B_d)) + d.fusedmm_bwd(V, A_d, B_d, G_d)
    torch.cuda.synchronize()
    d.close()
    want = expected(S, vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        x = x.double().cpu().numpy()
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


@pytest.mark.parametrize("r", [64, 24])
def test_sparse_shifting_two_ranks_on_one_gpu(r):
    """The sparse-shifting algorithm: column slices of 32 and 12 (r = 64, 24),
    fmm_sddmm_acc / fmm_spmm / fmm_spmm_t_acc per block row and phase."""
    import dist15d_ranks
    seed = 41 + r
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(2, seed, r, use_gpu=True, body="sparse_rank_main")
    got = assemble_slices(res, 2, S, r)
    want = expected(S, vals, A, B, G)[:2]
    for name, x, y in zip(("out", "out_t"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


def test_replicated_grid_four_ranks_on_one_gpu():
    """Algorithm 1 with replication factor 2 on a 2 x 2 grid: four gloo ranks
    on the one GPU, A all-gathered and the FusedMMA output and dA
    reduce-scattered along each fiber (staged through host memory)."""
    import dist15d_ranks
    seed, r = 71, 32
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(4, seed, r, use_gpu=True, c=2)
    got = assemble(res, 4, S, r)
    want = expected(S, vals, A, B, G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


@pytest.mark.parametrize("world,c", [(2, 1), (4, 2)])
def test_replication_reuse_on_one_gpu(world, c):
    """FusedMMA by replication reuse (fmm_sddmm per A block held, then
    fmm_spmm / fmm_spmm_acc into the travelling output blocks)."""
    import dist15d_ranks
    seed, r = 81 + world, 32
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(world, seed, r, use_gpu=True, body="reuse_rank_main", c=c)
    out = np.zeros((S.m, r))
    for k in range(world):
        r0, r1 = res[f"bounds{k}"]
        out[r0:r1] = res[k]["out"]
    assert np.all(np.isfinite(out))
    assert rel(out, expected(S, vals, A, B, G)[0]) <= 1e-5


def test_replicated_grid_bf16_on_one_gpu():
    """BF16 A and B on a 2 x 2 grid with the library's kernels: blocks
    gathered and shifted as raw bytes, FP32 outputs against the oracle on
    the BF16-rounded inputs within the FP32 bar."""
    import torch
    import dist15d_ranks
    seed, r = 91, 64
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(4, seed, r, use_gpu=True, c=2, bf16=True)
    got = assemble(res, 4, S, r)
    rnd = lambda X: torch.from_numpy(X).to(torch.bfloat16).float().numpy()  # noqa: E731
    want = expected(S, vals, rnd(A), rnd(B), G)
    for name, x, y in zip(("out", "out_t", "dA", "dB", "ds"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name


def test_sparse_shifting_replicated_grid_on_one_gpu():
    """Sparse shifting on a 2 x 2 grid with the library's kernels: B
    all-gathered along each fiber, block rows circulating in each layer,
    FusedMMB reduce-scattered along the fiber."""
    import dist15d_ranks
    seed, r = 97, 64
    S, vals, A, B, G = dist15d_ranks.problem(seed, r=r)
    res = run_ranks(4, seed, r, use_gpu=True, body="sparse_rank_main", c=2)
    got = assemble_slices(res, 4, S, r)
    want = expected(S, vals, A, B, G)[:2]
    for name, x, y in zip(("out", "out_t"), got, want):
        assert np.all(np.isfinite(x)), name
        assert rel(x, y) <= 1e-5, name
