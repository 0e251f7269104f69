"""GPU parity: every C-ABI call against the FP64 oracle, element by element.

Sizes span several thread blocks and a ragged tail; patterns cover empty
rows, duplicate and unsorted columns, hub rows and hub columns (split into
chunks), and r both on the vectorised path (32, 64, 128, 256) and on the
generic path (odd r, misaligned pointers).
"""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import (absolute, assert_close, deg_max, host64, oracle_all, relF,
                          upload)
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def pattern(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "er":
        return wl.er_exact_degree(700, 650, 32, rng), {}
    if kind == "irregular":
        return wl.random_csr(900, 650, rng, mean_deg=7, empty_frac=0.2, dup_frac=0.15,
                             unsorted=True), {}
    if kind == "hubs":
        S = wl.random_csr(600, 500, rng, mean_deg=5, empty_frac=0.1,
                          hubs=((3, 2500), (77, 700), (599, 130)))
        # a hub column too: 400 extra nonzeros in column 11, spread over rows
        rows = np.sort(rng.integers(0, 600, 400))
        deg = S.degrees().copy()
        np.add.at(deg, rows, 1)
        rp = np.zeros(601, np.int64); np.cumsum(deg, out=rp[1:])
        ci = np.empty(rp[-1], np.int32)
        extra = np.bincount(rows, minlength=600)
        for i in range(600):
            a, b = S.row_ptr[i], S.row_ptr[i + 1]
            ci[rp[i]:rp[i] + (b - a)] = S.col_idx[a:b]
            ci[rp[i] + (b - a):rp[i + 1]] = 11
        return wl.CSR(600, 500, rp.astype(np.int32), ci), {"split_nnz": 64}
    raise ValueError(kind)


def run_all(S, opts, r, dtype, seed, check_bf16_vs_f32=False):
    rng = np.random.default_rng(seed)
    vals = rng.uniform(0.0, 1.0, S.nnz).astype(np.float32)
    A = (rng.standard_normal((S.m, r)) / np.sqrt(r)).astype(np.float32)
    B = (rng.standard_normal((S.n, r)) / np.sqrt(r)).astype(np.float32)
    G = rng.standard_normal((S.m, r)).astype(np.float32)
    Gn = rng.standard_normal((S.n, r)).astype(np.float32)
    v_in = rng.standard_normal(S.nnz).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    Gt, Gnt = torch.from_numpy(G).cuda(), torch.from_numpy(Gn).cuda()
    v_t = torch.from_numpy(v_in).cuda()
    from paper_2203_07673_gb300 import fmm
    plan = fmm.Plan(rp, ci, S.n, r, dtype, **opts)
    got = dict(
        fusedmm=fmm.fusedmm(plan, vt, At, Bt),
        fusedmm_t=fmm.fusedmm_t(plan, vt, At, Bt),
        sddmm=fmm.sddmm(plan, vt, At, Bt),
        spmm=fmm.spmm(plan, v_t, Bt),
        spmm_t=fmm.spmm_t(plan, v_t, At),
        bwd=fmm.fusedmm_bwd(plan, vt, At, Bt, Gt),
        t_bwd=fmm.fusedmm_t_bwd(plan, vt, At, Bt, Gnt),
    )
    unfused = fmm.spmm(plan, got["sddmm"], Bt)
    torch.cuda.synchronize()
    A64, B64, s64 = host64(At), host64(Bt), vals.astype(np.float64)
    ref = oracle_all(S, s64, A64, B64, G, Gn)
    mag = oracle_all(S, absolute(s64), np.abs(A64), np.abs(B64), np.abs(G), np.abs(Gn))
    ref["spmm"] = oracle.spmm(S.row_ptr, S.col_idx, v_in, B64, S.n)
    ref["spmm_t"] = oracle.spmm_t(S.row_ptr, S.col_idx, v_in, A64, S.n)
    mag["spmm"] = oracle.spmm(S.row_ptr, S.col_idx, np.abs(v_in), np.abs(B64), S.n)
    mag["spmm_t"] = oracle.spmm_t(S.row_ptr, S.col_idx, np.abs(v_in), np.abs(A64), S.n)
    dm = deg_max(S)
    errs = {}
    for k in ("fusedmm", "fusedmm_t", "sddmm", "spmm", "spmm_t"):
        errs[k] = assert_close(k, got[k], ref[k], mag[k], r, dm)
    for k in ("bwd", "t_bwd"):
        for t, name in enumerate(("dA", "dB", "ds")):
            errs[f"{k}.{name}"] = assert_close(f"{k}.{name}", got[k][t], ref[k][t], mag[k][t],
                                               2 * r, dm)
    # the unfused SDDMM -> SpMM chain computes the same FusedMMA
    errs["unfused"] = assert_close("unfused", unfused, ref["fusedmm"], mag["fusedmm"], r + 1, dm)
    if check_bf16_vs_f32:
        ref32 = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A, B, S.n)
        e = relF(got["fusedmm"].cpu().double().numpy(), ref32)
        assert e <= 2e-2, e
        errs["fusedmm_vs_f32_samples"] = e
    plan.close()
    return errs


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [32, 64, 128, 256, 5, 24, 100, 520])
@pytest.mark.parametrize("kind", ["er", "irregular", "hubs"])
def test_parity_all_ops(kind, r, dtype):
    S, opts = pattern(kind, 1000 + r)
    run_all(S, opts, r, dtype, seed=r, check_bf16_vs_f32=(dtype == torch.bfloat16))


@pytest.mark.parametrize("variant", [114, 118, 222, 224, 441, 442, 214, 124, 112, 122, 212, 221,
                                     1041, 1042, 1081, 1082])
@pytest.mark.parametrize("split_nnz", [16, 0])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [32, 128, 256])
def test_kernel_variants(r, dtype, split_nnz, variant):
    S, _ = pattern("hubs", 7)
    run_all(S, {"split_nnz": split_nnz, "variant": variant}, r, dtype, seed=3)


# the register-ring (2xxxx, 3xxxx), bulk-staged (4xxxx) and streaming (5xxxx)
# forward passes
PIPELINED_AND_BULK = [22212, 23212, 22412, 32212, 24221, 34221, 23421, 23241,
                      44042, 43082, 44041, 44081, 52212, 52412, 54211]


@pytest.mark.parametrize("variant", PIPELINED_AND_BULK)
@pytest.mark.parametrize("split_nnz", [16, 0])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [32, 64, 128, 256])
def test_pipelined_and_bulk_variants(r, dtype, split_nnz, variant):
    S, _ = pattern("hubs", 7)
    run_all(S, {"split_nnz": split_nnz, "variant": variant}, r, dtype, seed=3)


@pytest.mark.parametrize("variant", PIPELINED_AND_BULK)
def test_pipelined_and_bulk_report_no_timeout(variant):
    """A bulk-staged pass that gave up a bounded wait sets the plan's error
    word; a normal run leaves it clear (fmm_plan_status returns FMM_OK)."""
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("er", 11)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((S.m, 64)).astype(np.float32)
    B = rng.standard_normal((S.n, 64)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, None, A, B, torch.bfloat16)
    plan = fmm.Plan(rp, ci, S.n, 64, torch.bfloat16, variant=variant)
    for _ in range(3):
        fmm.fusedmm(plan, None, At, Bt)
        fmm.fusedmm_t(plan, None, At, Bt)
    plan.status()
    plan.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [16, 32, 128])
def test_exact_small_integers_bitwise(r, dtype):
    # |x| <= 4, r <= 128, degree <= ~40: every partial sum is an integer below
    # 2^24, so float32 arithmetic is exact in any order: results must be
    # bitwise equal to the oracle's.
    from paper_2203_07673_gb300 import fmm
    rng = np.random.default_rng(r)
    S = wl.random_csr(300, 200, rng, mean_deg=8, empty_frac=0.2, dup_frac=0.2, unsorted=True,
                      hubs=((7, 40),))
    vals = wl.small_ints(S.nnz, 2, rng)
    A = wl.small_ints((300, r), 2, rng)
    B = wl.small_ints((200, r), 2, rng)
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=16)
    out = fmm.fusedmm(plan, vt, At, Bt).cpu().double().numpy()
    out_t = fmm.fusedmm_t(plan, vt, At, Bt).cpu().double().numpy()
    v = fmm.sddmm(plan, vt, At, Bt).cpu().double().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    assert np.array_equal(out, oracle.fusedmm(S.row_ptr, S.col_idx, vals, A64, B64, S.n))
    assert np.array_equal(out_t, oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A64, B64, S.n))
    assert np.array_equal(v, oracle.sddmm(S.row_ptr, S.col_idx, vals, A64, B64, S.n))
    G = wl.small_ints((300, r), 1, rng)
    dA, dB, ds = fmm.fusedmm_bwd(plan, vt, At, Bt, torch.from_numpy(G).cuda())
    eA, eB, es = oracle.fusedmm_grad(S.row_ptr, S.col_idx, vals, A64, B64, G, S.n)
    assert np.array_equal(dA.cpu().double().numpy(), eA)
    assert np.array_equal(dB.cpu().double().numpy(), eB)
    assert np.array_equal(ds.cpu().double().numpy(), es)


def test_deterministic_across_calls_and_plans():
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("hubs", 5)
    rng = np.random.default_rng(0)
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    A = rng.standard_normal((S.m, 128)).astype(np.float32)
    B = rng.standard_normal((S.n, 128)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B)
    p1 = fmm.Plan(rp, ci, S.n, 128, split_nnz=64)
    p2 = fmm.Plan(rp, ci, S.n, 128, split_nnz=64)
    for f in (fmm.fusedmm, fmm.fusedmm_t):
        a, b, c = f(p1, vt, At, Bt), f(p1, vt, At, Bt), f(p2, vt, At, Bt)
        assert torch.equal(a, b) and torch.equal(a, c)


def test_empty_and_degenerate_shapes():
    from paper_2203_07673_gb300 import fmm
    dev = "cuda"
    # nnz = 0: outputs are zero-filled
    rp = torch.zeros(6, dtype=torch.int32, device=dev)
    ci = torch.zeros(0, dtype=torch.int32, device=dev)
    A = torch.randn(5, 32, device=dev); B = torch.randn(7, 32, device=dev)
    p = fmm.Plan(rp, ci, 7, 32)
    out = torch.full((5, 32), 7.0, device=dev)
    fmm.fusedmm(p, None, A, B, out=out)
    assert not out.any()
    out_t = torch.full((7, 32), 7.0, device=dev)
    fmm.fusedmm_t(p, None, A, B, out=out_t)
    assert not out_t.any()
    assert fmm.sddmm(p, None, A, B).numel() == 0
    dA, dB, ds = fmm.fusedmm_bwd(p, None, A, B, torch.randn(5, 32, device=dev))
    assert not dA.any() and not dB.any()
    # m = 0
    p0 = fmm.Plan(torch.zeros(1, dtype=torch.int32, device=dev), ci, 7, 32)
    assert fmm.fusedmm(p0, None, torch.empty(0, 32, device=dev), B).shape == (0, 32)
    assert not fmm.fusedmm_t(p0, None, torch.empty(0, 32, device=dev), B).any()
    # n = 0 with rows
    pn = fmm.Plan(torch.zeros(4, dtype=torch.int32, device=dev), ci, 0, 8)
    assert not fmm.fusedmm(pn, None, torch.randn(3, 8, device=dev),
                           torch.empty(0, 8, device=dev)).any()
    # one long row split into many chunks, r = 1 (generic path)
    S = wl.CSR(1, 5000, np.array([0, 5000], np.int32), np.arange(5000, dtype=np.int32))
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 1)).astype(np.float32)
    b = rng.standard_normal((5000, 1)).astype(np.float32)
    s = rng.uniform(0, 1, 5000).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, s, a, b)
    p1 = fmm.Plan(rp, ci, 5000, 1, split_nnz=300)
    got = fmm.fusedmm(p1, vt, At, Bt).cpu().double().numpy()
    exp = a.astype(np.float64) * np.sum(s.astype(np.float64) * b[:, 0].astype(np.float64) ** 2)
    assert abs(got[0, 0] - exp[0, 0]) <= 1e-5 * abs(exp[0, 0])


def test_misaligned_pointers_take_generic_path():
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("irregular", 3)
    rng = np.random.default_rng(1)
    r = 32
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    rp, ci, vt, _, _ = upload(S, vals, A, B)
    # views at a 4-byte offset: not 16-byte aligned
    Abuf = torch.zeros(S.m * r + 1, device="cuda"); Abuf[1:] = torch.from_numpy(A).reshape(-1).cuda()
    Bbuf = torch.zeros(S.n * r + 1, device="cuda"); Bbuf[1:] = torch.from_numpy(B).reshape(-1).cuda()
    At, Bt = Abuf[1:].view(S.m, r), Bbuf[1:].view(S.n, r)
    assert At.data_ptr() % 16 != 0
    plan = fmm.Plan(rp, ci, S.n, r)
    got = fmm.fusedmm(plan, vt, At, Bt)
    ref = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A, B, S.n)
    mag = oracle.fusedmm(S.row_ptr, S.col_idx, vals, np.abs(A), np.abs(B), S.n)
    assert_close("misaligned fusedmm", got, ref, mag, r, deg_max(S))


@pytest.mark.parametrize("variant", [32212, 22212, 52212])
def test_ring_pass_needs_32_byte_rows(variant):
    """The register-ring pass loads gathered rows 32 bytes at a time: with
    A and B 16-byte but not 32-byte aligned (BF16, r = 64) the call takes the
    team kernel; aligned or not, FusedMMA and FusedMMB match the oracle."""
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("hubs", 5)
    rng = np.random.default_rng(2)
    r = 64
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    vals = rng.uniform(0.5, 1.5, S.nnz).astype(np.float32)
    rp, ci, vt, _, _ = upload(S, vals, A, B)
    Ab = torch.from_numpy(A).to(torch.bfloat16)
    Bb = torch.from_numpy(B).to(torch.bfloat16)
    A64, B64 = Ab.double().numpy(), Bb.double().numpy()
    ref = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A64, B64, S.n)
    mag = oracle.fusedmm(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n)
    ref_t = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A64, B64, S.n)
    mag_t = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n)
    plan = fmm.Plan(rp, ci, S.n, r, torch.bfloat16, variant=variant)
    for off in (0, 8):   # bf16 elements: 0 or 16 bytes past a 512-byte boundary
        Abuf = torch.zeros(S.m * r + 16, dtype=torch.bfloat16, device="cuda")
        Bbuf = torch.zeros(S.n * r + 16, dtype=torch.bfloat16, device="cuda")
        Abuf[off:off + S.m * r] = Ab.reshape(-1).cuda()
        Bbuf[off:off + S.n * r] = Bb.reshape(-1).cuda()
        At = Abuf[off:off + S.m * r].view(S.m, r)
        Bt = Bbuf[off:off + S.n * r].view(S.n, r)
        assert (At.data_ptr() % 32 == 0) == (off == 0) and At.data_ptr() % 16 == 0
        assert_close(f"ring fusedmm off={off}", fmm.fusedmm(plan, vt, At, Bt), ref, mag, r,
                     deg_max(S))
        assert_close(f"ring fusedmm_t off={off}", fmm.fusedmm_t(plan, vt, At, Bt), ref_t, mag_t,
                     r, int(np.bincount(S.col_idx, minlength=S.n).max()))
    plan.close()


def test_all_ones_pattern_matches_dense_gemm():
    # dense pattern, s = 1: FusedMMA = A (B^T B), FusedMMB = B (A^T A)
    from paper_2203_07673_gb300 import fmm
    m = n = 512
    r = 64
    rp = torch.arange(0, (m + 1) * n, n, dtype=torch.int32, device="cuda")
    ci = torch.arange(n, dtype=torch.int32, device="cuda").repeat(m)
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(m, r, device="cuda", generator=g) / 8
    B = torch.randn(n, r, device="cuda", generator=g) / 8
    plan = fmm.Plan(rp, ci, n, r)
    out = fmm.fusedmm(plan, None, A, B).double()
    out_t = fmm.fusedmm_t(plan, None, A, B).double()
    A64, B64 = A.double(), B.double()
    e1 = (out - A64 @ (B64.T @ B64)).norm() / (A64 @ (B64.T @ B64)).norm()
    e2 = (out_t - B64 @ (A64.T @ A64)).norm() / (B64 @ (A64.T @ A64)).norm()
    assert e1 <= 1e-5 and e2 <= 1e-5, (float(e1), float(e2))


def test_malformed_pattern_is_rejected():
    from paper_2203_07673_gb300 import fmm
    rp = torch.tensor([0, 2, 1, 3], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    assert fmm.validate(rp, ci, 4) == -(2 + 2)
    with pytest.raises(fmm.FmmError) as ei:
        fmm.Plan(rp, ci, 4, 32)
    assert ei.value.status == fmm.FMM_EINVAL
    rp = torch.tensor([0, 2, 3], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0, 9, 2], dtype=torch.int32, device="cuda")
    assert fmm.validate(rp, ci, 4) == 1
    with pytest.raises(fmm.FmmError):
        fmm.Plan(rp, ci, 4, 32)
    ok = torch.tensor([0, 2, 3], dtype=torch.int32, device="cuda")
    assert fmm.validate(ok, torch.tensor([0, 3, 2], dtype=torch.int32, device="cuda"), 4) == -1


def test_no_transpose_plan():
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("er", 1)
    rp, ci, vt, At, Bt = upload(S, None, np.ones((S.m, 32), np.float32),
                                np.ones((S.n, 32), np.float32))
    plan = fmm.Plan(rp, ci, S.n, 32, transpose=False)
    fmm.fusedmm(plan, None, At, Bt)
    with pytest.raises(fmm.FmmError) as ei:
        fmm.fusedmm_t(plan, None, At, Bt)
    assert ei.value.status == fmm.FMM_EUNSUPPORTED
    assert plan.info()["max_col_nnz"] == -1


def test_plan_info_reports_schedule():
    from paper_2203_07673_gb300 import fmm
    S, opts = pattern("hubs", 2)
    rp, ci, *_ = upload(S, None, np.zeros((S.m, 8), np.float32), np.zeros((S.n, 8), np.float32))
    info = fmm.Plan(rp, ci, S.n, 64, **opts).info()
    deg = S.degrees()
    cdeg = np.bincount(S.col_idx, minlength=S.n)
    assert info["max_row_nnz"] == deg.max() and info["max_col_nnz"] == cdeg.max()
    assert info["split_rows"] == (deg > 64).sum() and info["split_cols"] == (cdeg > 64).sum()
    assert info["row_chunks"] == int(np.ceil(deg[deg > 64] / 64).sum())


@pytest.mark.parametrize("offset", [0, 1], ids=["aligned", "unaligned"])
def test_value_permutation_large_unaligned(offset):
    """FusedMMB gathers the values of S into the order of S^T before its
    pass (four per thread in blocks of 1024); over 2^20 nonzeros, a ragged
    tail and values that are not 16-byte aligned, the result must match the
    oracle, and registered values must give the same bits."""
    from paper_2203_07673_gb300 import fmm
    rng = np.random.default_rng(11 + offset)
    m, n = 40000, 30000
    S = wl.random_csr(m, n, rng, mean_deg=27, empty_frac=0.02, unsorted=True, hubs=((2, 5000),))
    assert S.nnz >= 1 << 20 and (offset or S.nnz % 4 != 0)   # a ragged tail when aligned
    r = 8
    A = rng.standard_normal((m, r)).astype(np.float32)
    B = rng.standard_normal((n, r)).astype(np.float32)
    vals = rng.uniform(0.5, 1.5, S.nnz).astype(np.float32)
    rp, ci, _, At, Bt = upload(S, None, A, B)
    buf = torch.zeros(S.nnz + 1, device="cuda")
    buf[offset:offset + S.nnz] = torch.from_numpy(vals).cuda()
    vt = buf[offset:offset + S.nnz]
    plan = fmm.Plan(rp, ci, n, r)
    got = fmm.fusedmm_t(plan, vt, At, Bt)
    ref = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A, B, n)
    mag = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, np.abs(A), np.abs(B), n)
    cdeg = int(np.bincount(S.col_idx, minlength=n).max())
    assert_close("fusedmm_t (staged values)", got, ref, mag, r, cdeg)
    # registered values take the same two passes
    plan.set_values(vt)
    assert torch.equal(fmm.fusedmm_t(plan, vt, At, Bt), got)
    plan.set_values(None)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [32, 64, 128, 256])
@pytest.mark.parametrize("staged,team", [(1041, 112), (1081, 112), (1042, 212), (1082, 212)])
def test_staged_pass_equals_team_pass_bitwise(r, dtype, staged, team):
    """The staged pass (gathered rows in flight in shared memory) adds the
    same products in the same order as the team kernel with one group and
    two nonzeros per batch: FusedMM, FusedMMB, SDDMM and SpMM agree bit for
    bit, with long rows split and empty rows present."""
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("hubs", 11)
    rng = np.random.default_rng(r)
    vals = rng.uniform(0.0, 1.0, S.nnz).astype(np.float32)
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    v_in = torch.from_numpy(rng.standard_normal(S.nnz).astype(np.float32)).cuda()
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    out = {}
    for code in (staged, team):
        plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=48, variant=code)
        out[code] = (fmm.fusedmm(plan, vt, At, Bt), fmm.fusedmm_t(plan, vt, At, Bt),
                     fmm.sddmm(plan, vt, At, Bt), fmm.spmm(plan, v_in, Bt),
                     fmm.spmm_t(plan, v_in, At), fmm.fusedmm(plan, None, At, Bt))
        plan.close()
    for x, y in zip(out[staged], out[team]):
        assert torch.equal(x, y)


def test_rows_without_nonzeros_are_zeroed():
    """Outputs are overwritten, rows without nonzeros included: outputs filled
    with NaN beforehand must come back with exact zeros on those rows
    (FusedMM, FusedMMB, SpMM, both gradients, GAT, team and staged passes,
    vector and generic paths), and match the oracle elsewhere."""
    from paper_2203_07673_gb300 import fmm
    S = wl.random_csr(900, 1400, np.random.default_rng(5), mean_deg=5, empty_frac=0.2,
                      dup_frac=0.1, unsorted=True)
    deg, cdeg = S.degrees(), np.bincount(S.col_idx, minlength=S.n)
    assert (deg == 0).sum() > 50 and (cdeg == 0).sum() > 20
    rng = np.random.default_rng(2)
    for r, code in ((32, 0), (128, 0), (64, 1082), (24, 0), (64, 32212), (64, 44042),
                    (64, 52212), (128, 54211)):
        A = rng.standard_normal((S.m, r)).astype(np.float32)
        B = rng.standard_normal((S.n, r)).astype(np.float32)
        vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
        rp, ci, vt, At, Bt = upload(S, vals, A, B)
        plan = fmm.Plan(rp, ci, S.n, r, variant=code)
        nan = lambda *shape: torch.full(shape, float("nan"), device="cuda")  # noqa: E731
        out, out_t = nan(S.m, r), nan(S.n, r)
        fmm.fusedmm(plan, vt, At, Bt, out=out)
        fmm.fusedmm_t(plan, vt, At, Bt, out=out_t)
        sp = fmm.spmm(plan, vt, Bt, out=nan(S.m, r))
        G = torch.randn(S.m, r, device="cuda")
        dA, dB, ds = fmm.fusedmm_bwd(plan, vt, At, Bt, G)
        for name, t, empty in (("fusedmm", out, deg == 0), ("fusedmm_t", out_t, cdeg == 0),
                               ("spmm", sp, deg == 0), ("dA", dA, deg == 0),
                               ("dB", dB, cdeg == 0)):
            h = t.cpu().numpy()
            assert np.all(h[empty] == 0.0), name
            assert np.all(np.isfinite(h)), name
        ref = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A, B, S.n)
        assert relF(out.double().cpu().numpy(), ref) <= 1e-5
        if r % 8 == 0:
            heads = 2
            f = torch.randn(S.m, heads, device="cuda")
            g = torch.randn(S.n, heads, device="cuda")
            go = fmm.gat_forward(plan, heads, vt, f, g, Bt, 0.2, out=nan(S.m, r))
            h = go.cpu().numpy()
            assert np.all(h[deg == 0] == 0.0) and np.all(np.isfinite(h))
        plan.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("variant", [0, 212, 1042, 32212, 44042, 52212])
@pytest.mark.parametrize("r", [32, 128, 24])
def test_accumulating_calls_add_to_the_output(r, variant, dtype):
    """fmm_fusedmm_acc / _t_acc / _bwd_acc and fmm_sddmm_acc / _spmm_acc /
    _spmm_t_acc add the pass to what the outputs hold (split rows and
    columns included): acc(X0) equals X0 + the plain call, bit for bit where
    X0 = 0, within rounding otherwise."""
    from paper_2203_07673_gb300 import fmm
    S, _ = pattern("hubs", 5)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=64, variant=variant)
    G = torch.randn(S.m, r, device="cuda")
    ref = fmm.fusedmm(plan, vt, At, Bt)
    ref_t = fmm.fusedmm_t(plan, vt, At, Bt)
    rdA, rdB, rds = fmm.fusedmm_bwd(plan, vt, At, Bt, G)
    z = lambda *s: torch.zeros(s, device="cuda")  # noqa: E731
    assert torch.equal(fmm.fusedmm_acc(plan, vt, At, Bt, z(S.m, r)), ref)
    assert torch.equal(fmm.fusedmm_t_acc(plan, vt, At, Bt, z(S.n, r)), ref_t)
    dA, dB, ds = fmm.fusedmm_bwd_acc(plan, vt, At, Bt, G, z(S.m, r), z(S.n, r), z(S.nnz))
    assert torch.equal(dA, rdA) and torch.equal(dB, rdB) and torch.equal(ds, rds)
    v = fmm.sddmm(plan, vt, At, Bt)
    assert torch.equal(fmm.sddmm_acc(plan, vt, At, Bt, z(S.nnz)), v)
    assert torch.equal(fmm.spmm_acc(plan, v, Bt, z(S.m, r)), fmm.spmm(plan, v, Bt))
    assert torch.equal(fmm.spmm_t_acc(plan, v, At, z(S.n, r)), fmm.spmm_t(plan, v, At))
    V0 = torch.randn(S.nnz, device="cuda")
    err = (fmm.sddmm_acc(plan, vt, At, Bt, V0.clone()) - (V0 + v)).abs().max().item()
    assert err <= 1e-5 * max(1.0, (V0 + v).abs().max().item()), err
    X0, Y0 = torch.randn(S.m, r, device="cuda"), torch.randn(S.n, r, device="cuda")
    got = fmm.fusedmm_acc(plan, vt, At, Bt, X0.clone())
    got_t = fmm.fusedmm_t_acc(plan, vt, At, Bt, Y0.clone())
    # the vector passes add X0 to the finished row (one rounding, as X0 +
    # ref); the generic pass starts its sum from X0 (another order), so the
    # difference is rounding-sized, far below a missing X0 or term
    for g, w in ((got, X0 + ref), (got_t, Y0 + ref_t)):
        err = (g - w).abs().max().item()
        assert err <= 1e-5 * max(1.0, w.abs().max().item()), err
    plan.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_tune_plan_on_the_gpu_keeps_results(dtype):
    """tune_plan times candidates and the plan's own codes on its operands,
    sets the fastest per side, and the tuned plan still matches the oracle
    (forward, transpose and backward)."""
    from paper_2203_07673_gb300 import autotune
    S, _ = pattern("hubs", 13)
    rng = np.random.default_rng(13)
    r = 64
    vals = rng.uniform(0.0, 1.0, S.nnz).astype(np.float32)
    A = (rng.standard_normal((S.m, r)) / np.sqrt(r)).astype(np.float32)
    B = (rng.standard_normal((S.n, r)) / np.sqrt(r)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    from paper_2203_07673_gb300 import fmm
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=64)
    G = torch.randn(S.m, r, device="cuda")
    res = autotune.tune_plan(plan, vt, At, Bt, G, candidates=(112, 212, 32212), iters=2)
    info = plan.info()
    assert (info["variant"], info["variant_t"]) == (res["variant"], res["variant_t"])
    assert res["variant"] in res["ms"] and res["variant_t"] in res["ms_t"]
    A64, B64 = At.double().cpu().numpy(), Bt.double().cpu().numpy()
    ref = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A64, B64, S.n)
    mag = oracle.fusedmm(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n)
    assert_close("tuned fusedmm", fmm.fusedmm(plan, vt, At, Bt), ref, mag, r, deg_max(S))
    ref_t = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, A64, B64, S.n)
    mag_t = oracle.fusedmm_t(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n)
    assert_close("tuned fusedmm_t", fmm.fusedmm_t(plan, vt, At, Bt), ref_t, mag_t, r, deg_max(S))
    plan.close()
