"""Parity at the full workload sizes, in the plan configuration bench.py
times, on sampled rows and columns the oracle computes exactly.

A sampled row i of FusedMMA (and dA_i, ds of row i) depends only on the
nonzeros of row i; a sampled column j of FusedMMB (and dB_j) only on the
nonzeros of column j.  So each check runs the oracle on the sub-pattern of
the sampled rows (or columns) and compares element by element.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, cols_problem, relF, rows_problem
from paper_2203_07673_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _cmp(name, got, ref, mag, terms, tol=1e-5):
    got = np.asarray(got, np.float64)
    bound = 2.0 * terms * U32 * mag + 1e-30
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{name}: {bad.sum()} elements over the rounding bound"
    e = relF(got, ref)
    assert e <= tol, f"{name}: relF {e:.2e}"
    return e


def _sampled_fwd(w, dt, plan, vt, At, Bt, n_rows=384, n_cols=384, seed=0):
    from paper_2203_07673_gb300 import fmm
    S, r = w["S"], w["r"]
    out = fmm.fusedmm(plan, vt, At, Bt)
    out_t = fmm.fusedmm_t(plan, vt, At, Bt)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(S.m, n_rows, replace=False))
    rows[0] = int(np.argmax(S.degrees()))                  # the longest row too
    cols = np.sort(rng.choice(S.n, n_cols, replace=False))
    cols[0] = int(np.argmax(np.bincount(S.col_idx, minlength=S.n)))
    rows, cols = np.unique(rows), np.unique(cols)
    A64 = At[torch.from_numpy(np.unique(np.concatenate([rows]))).cuda()].double().cpu().numpy()
    vals = w["vals"]
    rp, ci, v, cused, _ = rows_problem(S, rows, vals)
    B_used = Bt[torch.from_numpy(cused).cuda()].double().cpu().numpy()
    ref = oracle.fusedmm(rp, ci, v, A64, B_used, len(cused))
    mag = oracle.fusedmm(rp, ci, None if v is None else np.abs(v), np.abs(A64),
                         np.abs(B_used), len(cused))
    deg = int(S.degrees().max())
    e1 = _cmp("FusedMMA rows", out[torch.from_numpy(rows).cuda()].double().cpu().numpy(),
              ref, mag, r + deg + 4)
    rp, ci, v, rused, _ = cols_problem(S, cols, vals)
    A_used = At[torch.from_numpy(rused).cuda()].double().cpu().numpy()
    B_c = Bt[torch.from_numpy(cols).cuda()].double().cpu().numpy()
    ref = oracle.fusedmm_t(rp, ci, v, A_used, B_c, len(cols))
    mag = oracle.fusedmm_t(rp, ci, None if v is None else np.abs(v), np.abs(A_used),
                           np.abs(B_c), len(cols))
    cdeg = int(np.bincount(S.col_idx, minlength=S.n).max())
    e2 = _cmp("FusedMMB cols", out_t[torch.from_numpy(cols).cuda()].double().cpu().numpy(),
              ref, mag, r + cdeg + 4)
    return e1, e2


def _upload(w, dt):
    S = w["S"]
    rp = torch.from_numpy(S.row_ptr).cuda()
    ci = torch.from_numpy(S.col_idx).cuda()
    vt = None if w["vals"] is None else torch.from_numpy(w["vals"]).cuda()
    At = torch.from_numpy(w["A"]).cuda().to(dt).contiguous()
    Bt = torch.from_numpy(w["B"]).cuda().to(dt).contiguous()
    return rp, ci, vt, At, Bt


def test_er_2p20_r128_f32_bench_configuration():
    from paper_2203_07673_gb300 import fmm
    w = wl.workload(2)
    rp, ci, vt, At, Bt = _upload(w, torch.float32)
    plan = fmm.Plan(rp, ci, w["S"].n, w["r"], torch.float32)   # as bench.py
    _sampled_fwd(w, torch.float32, plan, vt, At, Bt)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_zipf_rows_2p21x2p19_r64(dt):
    from paper_2203_07673_gb300 import fmm
    w = wl.workload(4)
    rp, ci, vt, At, Bt = _upload(w, dt)
    plan = fmm.Plan(rp, ci, w["S"].n, w["r"], dt)
    _sampled_fwd(w, dt, plan, vt, At, Bt, seed=1)


def test_rmat_2p22_r64_bf16_forward_backward():
    from paper_2203_07673_gb300 import fmm
    w = wl.workload(3)
    S, r = w["S"], w["r"]
    rp, ci, _, At, Bt = _upload(w, torch.bfloat16)
    ones = torch.ones(S.nnz, device="cuda")          # s = 1, gradient wanted
    plan = fmm.Plan(rp, ci, S.n, r, torch.bfloat16)
    w1 = dict(w, vals=None)
    _sampled_fwd(w1, torch.bfloat16, plan, None, At, Bt, seed=2)
    G = torch.randn(S.m, r, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    dA, dB, ds = fmm.fusedmm_bwd(plan, ones, At, Bt, G)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[int(np.argmax(S.degrees()))],
                                     rng.choice(S.m, 256, replace=False)]))
    cols = np.unique(np.concatenate([[int(np.argmax(np.bincount(S.col_idx, minlength=S.n)))],
                                     rng.choice(S.n, 256, replace=False)]))
    t = lambda idx: torch.from_numpy(np.asarray(idx)).cuda()
    # dA and ds of the sampled rows
    srp, sci, _, cused, nz = rows_problem(S, rows)
    A_r = At[t(rows)].double().cpu().numpy(); B_c = Bt[t(cused)].double().cpu().numpy()
    G_r = G[t(rows)].double().cpu().numpy()
    ref = oracle.fusedmm_grad(srp, sci, None, A_r, B_c, G_r, len(cused))
    mag = oracle.fusedmm_grad(srp, sci, None, np.abs(A_r), np.abs(B_c), np.abs(G_r), len(cused))
    deg = int(S.degrees().max())
    _cmp("dA rows", dA[t(rows)].double().cpu().numpy(), ref[0], mag[0], 2 * r + deg + 4)
    _cmp("ds of the rows", ds[t(nz)].double().cpu().numpy(), ref[2], mag[2], 2 * r + 4)
    # dB of the sampled columns
    srp, sci, _, rused, _ = cols_problem(S, cols)
    A_r = At[t(rused)].double().cpu().numpy(); B_c = Bt[t(cols)].double().cpu().numpy()
    G_r = G[t(rused)].double().cpu().numpy()
    ref = oracle.fusedmm_grad(srp, sci, None, A_r, B_c, G_r, len(cols))
    mag = oracle.fusedmm_grad(srp, sci, None, np.abs(A_r), np.abs(B_c), np.abs(G_r), len(cols))
    cdeg = int(np.bincount(S.col_idx, minlength=S.n).max())
    _cmp("dB cols", dB[t(cols)].double().cpu().numpy(), ref[1], mag[1], 2 * r + cdeg + 4)


def test_er_4096_r32_f32_every_output_element():
    """The small configuration (ER 4096 x 4096, 32 distinct columns per row,
    r = 32, FP32, s ~ U(0,1)) at its exact size: every element of FusedMMA,
    FusedMMB, SDDMM, the unfused SDDMM -> SpMM chain and both gradients
    against the oracle."""
    from paper_2203_07673_gb300 import fmm
    from parity_utils import absolute, assert_close, deg_max, oracle_all
    w = wl.workload(1)
    S, r = w["S"], w["r"]
    rp, ci, vt, At, Bt = _upload(w, torch.float32)
    plan = fmm.Plan(rp, ci, S.n, r, torch.float32)   # as bench.py would
    rng = np.random.default_rng(9)
    G = rng.standard_normal((S.m, r)).astype(np.float32)
    Gn = rng.standard_normal((S.n, r)).astype(np.float32)
    Gt, Gnt = torch.from_numpy(G).cuda(), torch.from_numpy(Gn).cuda()
    v = fmm.sddmm(plan, vt, At, Bt)
    got = dict(fusedmm=fmm.fusedmm(plan, vt, At, Bt), fusedmm_t=fmm.fusedmm_t(plan, vt, At, Bt),
               sddmm=v, unfused=fmm.spmm(plan, v, Bt),
               bwd=fmm.fusedmm_bwd(plan, vt, At, Bt, Gt),
               t_bwd=fmm.fusedmm_t_bwd(plan, vt, At, Bt, Gnt))
    s64, A64, B64 = w["vals"].astype(np.float64), w["A"].astype(np.float64), w["B"].astype(np.float64)
    ref = oracle_all(S, s64, A64, B64, G, Gn)
    mag = oracle_all(S, absolute(s64), np.abs(A64), np.abs(B64), np.abs(G), np.abs(Gn))
    dm = deg_max(S)
    for k in ("fusedmm", "fusedmm_t", "sddmm"):
        assert_close(k, got[k], ref[k], mag[k], r, dm)
    assert_close("unfused", got["unfused"], ref["fusedmm"], mag["fusedmm"], r + 1, dm)
    for k in ("bwd", "t_bwd"):
        for t, name in enumerate(("dA", "dB", "ds")):
            assert_close(f"{k}.{name}", got[k][t], ref[k][t], mag[k][t], 2 * r, dm)
    plan.close()


def test_batched_512_matrices_sampled():
    """The batched configuration at its full size, in the launch the bench
    times: 512 uneven matrices (half ER, half R-MAT, BF16 A and B, r in
    {32, 64, 128}), forward and backward each one persistent launch.  Sampled
    rows (FusedMMA, dA, ds) and columns (dB) of sampled matrices, the largest
    among them, against the oracle on the BF16-rounded inputs."""
    from paper_2203_07673_gb300 import fmm
    dev = torch.device("cuda")
    items = []
    for t, sp in enumerate(wl.batched_specs(512)):
        m = wl.batched_matrix_torch(sp, t, dev)
        r = m["r"]
        plan = fmm.Plan(m["row_ptr"], m["col_idx"], m["n"], r, torch.bfloat16,
                        split_nnz=1 << 30)
        g = torch.Generator(device=dev)
        g.manual_seed(7919 * t + 1)
        items.append(dict(plan=plan, vals=m["vals"], A=m["A"].bfloat16().contiguous(),
                          B=m["B"].bfloat16().contiguous(),
                          G=torch.randn(m["m"], r, device=dev, generator=g),
                          out=torch.empty(m["m"], r, device=dev),
                          dA=torch.empty(m["m"], r, device=dev),
                          dB=torch.empty(m["n"], r, device=dev),
                          ds=torch.empty(m["col_idx"].numel(), device=dev),
                          rp=m["row_ptr"], ci=m["col_idx"]))
    keys = ("plan", "vals", "A", "B", "out", "G", "dA", "dB", "ds")
    batch = fmm.Batch([{k: it[k] for k in keys} for it in items])
    batch.forward()
    batch.backward()
    torch.cuda.synchronize()

    rng = np.random.default_rng(4)
    nnz = [it["ci"].numel() for it in items]
    picked = sorted(set(rng.choice(len(items), 6, replace=False).tolist()) |
                    {int(np.argmax(nnz))})
    host = lambda x: x.detach().double().cpu().numpy()   # noqa: E731
    for t in picked:
        it = items[t]
        p = it["plan"]
        S = wl.CSR(p.m, p.n, it["rp"].cpu().numpy().astype(np.int32),
                   it["ci"].cpu().numpy().astype(np.int32))
        vals = host(it["vals"])
        A, B, G = host(it["A"]), host(it["B"]), host(it["G"])
        deg = int(S.degrees().max())
        cdeg = int(np.bincount(S.col_idx, minlength=S.n).max())
        rows = np.unique(np.concatenate([rng.choice(S.m, min(128, S.m), replace=False),
                                         [int(np.argmax(S.degrees()))]]))
        rp, ci, v, cused, idx = rows_problem(S, rows, vals)
        ref = oracle.fusedmm(rp, ci, v, A[rows], B[cused], len(cused))
        mag = oracle.fusedmm(rp, ci, np.abs(v), np.abs(A[rows]), np.abs(B[cused]), len(cused))
        _cmp(f"batch {t} FusedMMA rows", host(it["out"])[rows], ref, mag, p.r + deg + 4)
        dA_r, _, ds_r = oracle.fusedmm_grad(rp, ci, v, A[rows], B[cused], G[rows], len(cused))
        dA_m, _, ds_m = oracle.fusedmm_grad(rp, ci, np.abs(v), np.abs(A[rows]),
                                            np.abs(B[cused]), np.abs(G[rows]), len(cused))
        _cmp(f"batch {t} dA rows", host(it["dA"])[rows], dA_r, dA_m, 2 * p.r + deg + 4)
        _cmp(f"batch {t} ds", host(it["ds"])[idx], ds_r, ds_m, 2 * p.r + 4)
        cols = np.unique(np.concatenate([rng.choice(S.n, min(128, S.n), replace=False),
                                         [int(np.argmax(np.bincount(S.col_idx, minlength=S.n)))]]))
        rp, ci, v, rused, _ = cols_problem(S, cols, vals)
        _, dB_c, _ = oracle.fusedmm_grad(rp, ci, v, A[rused], B[cols], G[rused], len(cols))
        _, dB_m, _ = oracle.fusedmm_grad(rp, ci, np.abs(v), np.abs(A[rused]), np.abs(B[cols]),
                                         np.abs(G[rused]), len(cols))
        _cmp(f"batch {t} dB cols", host(it["dB"])[cols], dB_c, dB_m, 2 * p.r + cdeg + 4)
    batch.close()
    for it in items:
        it["plan"].close()


def test_windowed_value_permutation_exact():
    """Plans with more than two windows (2^23 S^T slots each) of nonzeros put
    the values of S into S^T order in two passes (scatter into windows, then
    gather inside a window).  With small-integer values and all-ones A and
    B, FusedMMB and SpMMB are exact integer column sums of S, so every
    element must equal the column sums bit for bit; per-call and registered
    values both take the windowed path."""
    from paper_2203_07673_gb300 import fmm
    dev = torch.device("cuda")
    g = wl._torch_gen(dev, 4242)
    m, n, deg, r = 600_000, 1 << 18, 30, 32
    rp, ci = wl.er_exact_degree_torch(m, n, deg, g, dev)
    nnz = ci.numel()
    assert nnz > 2 * (1 << 23)
    vals = (torch.arange(nnz, device=dev) % 7).float()
    A = torch.ones(m, r, device=dev)
    B = torch.ones(n, r, device=dev)
    plan = fmm.Plan(rp, ci, n, r)
    colsum = torch.bincount(ci.long(), weights=vals.double(), minlength=n)
    want_t = (colsum * r).float()[:, None].expand(n, r)
    assert torch.equal(fmm.fusedmm_t(plan, vals, A, B), want_t)
    assert torch.equal(fmm.spmm_t(plan, vals, A), colsum.float()[:, None].expand(n, r))
    plan.set_values(vals)
    assert torch.equal(fmm.fusedmm_t(plan, vals, A, B), want_t)
    # values changed after registration are taken from the new pointer
    vals2 = (torch.arange(nnz, device=dev) % 5).float()
    colsum2 = torch.bincount(ci.long(), weights=vals2.double(), minlength=n)
    assert torch.equal(fmm.fusedmm_t(plan, vals2, A, B), (colsum2 * r).float()[:, None].expand(n, r))
    plan.close()
