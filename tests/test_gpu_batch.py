"""Batched persistent launch: every item against its own per-matrix calls
(bitwise, same kernel variants) and against the FP64 oracle; forward and
backward replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, relF
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def batch_codes(r, dtype):
    """Variant codes the batch kernels run in every role at width r (the
    rule of fmm_batch.cu: at most 32 floats live per lane in the forward
    phase, 48 in the backward phase)."""
    es = 4 if dtype == torch.float32 else 2
    vecs = r * es // 16
    base = max(1, vecs // 32)
    ok = []
    for code in (112, 114, 122, 212, 214, 221):
        V, N, U = (code // 100) * base, (code // 10) % 10, code % 10
        if vecs % V:
            continue
        g = vecs // V
        E = V * (16 // es)
        if g & (g - 1) or g * N > 32 or 32 % (g * N):
            continue
        if E * (U + 2) <= 32 and E * (2 * U + 2) <= 48 and E * (U + 3) <= 48:
            ok.append(code)
    return ok


def make_items(dtype, seed=0, count=10, variants=None):
    from paper_2203_07673_gb300 import fmm
    rng = np.random.default_rng(seed)
    specs = wl.batched_specs(count, seed_index=50 + seed, rows_lo=60, rows_hi=3000)
    items, host = [], []
    for t, sp in enumerate(specs):
        m = wl.batched_matrix(sp, t, seed_index=50 + seed)
        S, r = m["S"], m["r"]
        rp = torch.from_numpy(S.row_ptr).cuda()
        ci = torch.from_numpy(S.col_idx).cuda()
        plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=1 << 30)
        if variants is not None:
            codes = [c for c in variants if c in batch_codes(r, dtype)]
            plan.set_variant(codes[t % len(codes)], codes[(t + 1) % len(codes)])
        vals = torch.from_numpy(m["vals"]).cuda()
        A = torch.from_numpy(m["A"]).cuda().to(dtype).contiguous()
        B = torch.from_numpy(m["B"]).cuda().to(dtype).contiguous()
        G = torch.from_numpy(rng.standard_normal((S.m, r)).astype(np.float32)).cuda()
        items.append(dict(plan=plan, vals=vals, A=A, B=B, G=G,
                          out=torch.full((S.m, r), np.nan, device="cuda"),
                          dA=torch.full((S.m, r), np.nan, device="cuda"),
                          dB=torch.full((S.n, r), np.nan, device="cuda"),
                          ds=torch.full((S.nnz,), np.nan, device="cuda"),
                          rp=rp, ci=ci))
        host.append(m)
    return items, host


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_batch_matches_per_matrix_calls_and_oracle(dtype):
    from paper_2203_07673_gb300 import fmm
    items, host = make_items(dtype, seed=1, variants=[112, 114, 122, 212, 214, 221])
    batch = fmm.Batch([{k: it[k] for k in ("plan", "vals", "A", "B", "out", "G", "dA", "dB", "ds")}
                       for it in items])
    batch.forward()
    batch.backward()
    torch.cuda.synchronize()
    for it, m in zip(items, host):
        p = it["plan"]
        # per-matrix calls with the same variants give the same bits
        # (only variants the batch kernels have were selected above)
        ref_out = fmm.fusedmm(p, it["vals"], it["A"], it["B"])
        dA, dB, ds = fmm.fusedmm_bwd(p, it["vals"], it["A"], it["B"], it["G"])
        torch.cuda.synchronize()
        assert torch.equal(it["out"], ref_out)
        assert torch.equal(it["dA"], dA) and torch.equal(it["dB"], dB) and torch.equal(it["ds"], ds)
        # and the oracle agrees
        S = m["S"]
        A64 = it["A"].double().cpu().numpy(); B64 = it["B"].double().cpu().numpy()
        G64 = it["G"].double().cpu().numpy(); s64 = m["vals"].astype(np.float64)
        exp = oracle.fusedmm(S.row_ptr, S.col_idx, s64, A64, B64, S.n)
        mag = oracle.fusedmm(S.row_ptr, S.col_idx, s64, np.abs(A64), np.abs(B64), S.n)
        deg = max(int(S.degrees().max()), int(np.bincount(S.col_idx, minlength=S.n).max()))
        got = it["out"].double().cpu().numpy()
        assert np.all(np.abs(got - exp) <= 2 * (m["r"] + deg + 4) * U32 * mag + 1e-30)
        assert relF(got, exp) <= 1e-5
        g = oracle.fusedmm_grad(S.row_ptr, S.col_idx, s64, A64, B64, G64, S.n)
        gm = oracle.fusedmm_grad(S.row_ptr, S.col_idx, s64, np.abs(A64), np.abs(B64),
                                 np.abs(G64), S.n)
        for name, x, e, mg in (("dA", it["dA"], g[0], gm[0]), ("dB", it["dB"], g[1], gm[1]),
                               ("ds", it["ds"], g[2], gm[2])):
            xx = x.double().cpu().numpy()
            assert np.all(np.abs(xx - e) <= 2 * (2 * m["r"] + deg + 4) * U32 * mg + 1e-30), name
            assert relF(xx, e) <= 1e-5, name
    batch.close()


def test_batch_cuda_graph_replay():
    from paper_2203_07673_gb300 import fmm
    items, _ = make_items(torch.bfloat16, seed=2, count=8)
    batch = fmm.Batch([{k: it[k] for k in ("plan", "vals", "A", "B", "out", "G", "dA", "dB", "ds")}
                       for it in items])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.forward(); batch.backward()          # warm-up outside the graph
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [(it["out"].clone(), it["dA"].clone(), it["dB"].clone(), it["ds"].clone())
             for it in items]
    for it in items:
        for k in ("out", "dA", "dB", "ds"):
            it[k].fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.forward()
        batch.backward()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for it, e in zip(items, eager):
            for k, x in zip(("out", "dA", "dB", "ds"), e):
                assert torch.equal(it[k], x), k
    batch.close()


def test_batch_rejects_split_rows_and_mixed_dtypes():
    from paper_2203_07673_gb300 import fmm
    rng = np.random.default_rng(0)
    S = wl.random_csr(50, 40, rng, mean_deg=3, hubs=((0, 600),))
    rp = torch.from_numpy(S.row_ptr).cuda(); ci = torch.from_numpy(S.col_idx).cuda()
    A = torch.randn(50, 32, device="cuda"); B = torch.randn(40, 32, device="cuda")
    out = torch.empty(50, 32, device="cuda")
    split = fmm.Plan(rp, ci, 40, 32, split_nnz=64)
    with pytest.raises(fmm.FmmError) as ei:
        fmm.Batch([dict(plan=split, A=A, B=B, out=out)])
    assert ei.value.status == fmm.FMM_EUNSUPPORTED
    p32 = fmm.Plan(rp, ci, 40, 32, split_nnz=1 << 30)
    p16 = fmm.Plan(rp, ci, 40, 32, torch.bfloat16, split_nnz=1 << 30)
    with pytest.raises(fmm.FmmError):
        fmm.Batch([dict(plan=p32, A=A, B=B, out=out),
                   dict(plan=p16, A=A.bfloat16(), B=B.bfloat16(), out=out)])
    # forward-only batch: backward is refused
    b = fmm.Batch([dict(plan=p32, A=A, B=B, out=out)])
    b.forward()
    with pytest.raises(fmm.FmmError):
        b.backward()
    torch.cuda.synchronize()
    assert relF(out.double().cpu().numpy(),
                oracle.fusedmm(S.row_ptr, S.col_idx, None, A.double().cpu().numpy(),
                               B.double().cpu().numpy(), 40)) <= 1e-5
