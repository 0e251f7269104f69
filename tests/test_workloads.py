"""Structure of the seeded synthetic inputs (no method arithmetic here)."""
import numpy as np

from paper_2203_07673_gb300 import workloads as wl


def _valid(S):
    rp = S.row_ptr.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == S.nnz and np.all(np.diff(rp) >= 0)
    assert S.col_idx.dtype == np.int32 and S.row_ptr.dtype == np.int32
    if S.nnz:
        assert S.col_idx.min() >= 0 and S.col_idx.max() < S.n


def _distinct_sorted(S):
    for i in range(S.m):
        seg = S.col_idx[S.row_ptr[i]:S.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_er_exact_degree():
    S = wl.er_exact_degree(300, 257, 32, wl.config_rng(1, 0))
    _valid(S)
    assert np.all(S.degrees() == 32)
    _distinct_sorted(S)
    S2 = wl.er_exact_degree(300, 257, 32, wl.config_rng(1, 0))
    assert np.array_equal(S.col_idx, S2.col_idx)      # seeded
    D = wl.er_exact_degree(10, 40, 30, wl.config_rng(1, 9))   # dense-ish branch
    _valid(D)
    assert np.all(D.degrees() == 30)
    _distinct_sorted(D)


def test_rmat_power_law():
    S = wl.rmat(12, 16, 0.57, 0.19, 0.19, 0.05, wl.config_rng(3, 0))
    _valid(S)
    assert S.m == S.n == 4096
    assert S.nnz <= 16 * 4096
    _distinct_sorted(S)
    deg = S.degrees()
    assert deg.max() > 20 * deg.mean()        # heavy-tailed
    F = wl.rmat(10, 16, 0.57, 0.19, 0.19, 0.05, wl.config_rng(3, 1), vertices=1000)
    _valid(F)
    assert F.m == 1000


def test_zipf_rows():
    S = wl.zipf_rows(4096, 2048, 150_000, 1.2, 512, wl.config_rng(4, 0))
    _valid(S)
    assert abs(S.nnz - 150_000) <= 150
    assert S.degrees().min() >= 1 and S.degrees().max() <= 512
    _distinct_sorted(S)


def test_random_csr_features():
    rng = np.random.default_rng(0)
    S = wl.random_csr(200, 50, rng, mean_deg=6, empty_frac=0.3, dup_frac=0.3,
                      unsorted=True, hubs=((5, 900),))
    _valid(S)
    deg = S.degrees()
    assert deg[5] == 900 and (deg == 0).sum() > 20
    seg = S.col_idx[S.row_ptr[5]:S.row_ptr[6]]
    assert np.unique(seg).size < seg.size     # duplicates present


def test_value_recipes():
    v = wl.half_steps(10000, 1.0, 5.0, wl.config_rng(4, 1))
    assert set(np.unique(v * 2).astype(int)) <= set(range(2, 11))
    x = wl.normal(2000, 64, 0.1, wl.config_rng(4, 2))
    assert abs(x.var() - 0.1) < 0.005 and x.dtype == np.float32


def test_small_workloads():
    w = wl.workload(1)
    assert w["S"].m == 4096 and w["S"].nnz == 4096 * 32 and w["A"].shape == (4096, 32)
    w = wl.workload(2, scale_rows=1 / 256)
    assert w["S"].m == 4096 and w["A"].shape == (4096, 128)
    w = wl.workload(3, scale_rows=1 / 256)
    assert w["vals"] is None and w["A"].shape[1] == 64
    w = wl.workload(4, scale_rows=1 / 256)
    assert w["S"].m == 8192 and w["S"].n == 2048
    specs = wl.batched_specs(16, scale_rows=0.01)
    assert len(specs) == 16 and {s["r"] for s in specs} <= {32, 64, 128}
    m0 = wl.batched_matrix(specs[1], 1)
    _valid(m0["S"])


def test_torch_generators_on_cpu():
    """The device generators of the batched and GAT inputs (run here on the
    CPU device): valid CSR, distinct sorted columns where the recipe says so,
    seeded, and the batched matrix of a spec has the spec's shape."""
    import torch
    g = wl._torch_gen("cpu", 5)
    rp, ci = wl.er_exact_degree_torch(300, 257, 32, g, "cpu")
    S = wl.CSR(300, 257, rp.numpy().astype(np.int32), ci.numpy().astype(np.int32))
    _valid(S)
    assert np.all(S.degrees() == 32)
    _distinct_sorted(S)
    rp, ci = wl.rmat_torch(10, 16 * 1000, 0.57, 0.19, 0.19, wl._torch_gen("cpu", 6), "cpu", 1000)
    R = wl.CSR(1000, 1000, rp.numpy().astype(np.int32), ci.numpy().astype(np.int32))
    _valid(R)
    _distinct_sorted(R)
    assert R.degrees().max() > 10 * R.degrees().mean()
    rp2, ci2 = wl.rmat_torch(10, 16 * 1000, 0.57, 0.19, 0.19, wl._torch_gen("cpu", 6), "cpu", 1000)
    assert torch.equal(rp, rp2) and torch.equal(ci, ci2)
    specs = wl.batched_specs(8, scale_rows=0.01)
    for t in (0, 1):
        m = wl.batched_matrix_torch(specs[t], t, "cpu")
        assert m["m"] == m["n"] == specs[t]["rows"] and m["r"] == specs[t]["r"]
        assert m["A"].shape == (m["m"], m["r"]) and m["vals"].numel() == m["col_idx"].numel()
        B = wl.CSR(m["m"], m["n"], m["row_ptr"].numpy().astype(np.int32),
                   m["col_idx"].numpy().astype(np.int32))
        _valid(B)
