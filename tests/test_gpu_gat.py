"""Graph-attention forward (Sec. VI-E) on the GPU against the FP64 oracle,
and registered values (fmm_plan_set_values).

Tolerance of the attention output: a score e = LeakyReLU(s (f + g)) is
rounded to a few ulp of |e|, so exp(e - max) carries a relative error of
about (4 |e|_max + 4) u; the softmax normaliser adds deg u and the
aggregation another deg u relative to sum_j alpha_ij |H_j|, which is the
oracle's output on |H|.  Each element must lie within
2 (8 |e|_max + 2 deg + 16) u times that magnitude (u = 2^-24), and the
relative Frobenius error within 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, relF, upload
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _graph(seed, m=700, hubs=((5, 1500),)):
    rng = np.random.default_rng(seed)
    return wl.random_csr(m, m, rng, mean_deg=9, empty_frac=0.1, dup_frac=0.05, unsorted=True,
                         hubs=hubs), rng


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("heads,rh", [(4, 32), (2, 32), (1, 64), (8, 16), (4, 8), (3, 8), (2, 12)])
def test_gat_forward_matches_oracle(heads, rh, dtype):
    from paper_2203_07673_gb300 import fmm
    S, rng = _graph(heads * 100 + rh)
    r = heads * rh
    H = (rng.standard_normal((S.n, r)) * 0.5).astype(np.float32)
    f = rng.standard_normal((S.m, heads)).astype(np.float32)
    g = rng.standard_normal((S.n, heads)).astype(np.float32)
    vals = rng.uniform(0.5, 1.5, S.nnz).astype(np.float32)
    rp, ci, vt, _, Ht = upload(S, vals, f, H, dtype)
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=256)   # the hub row is split: taken whole
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    slope = 0.2
    out = fmm.gat_forward(plan, heads, vt, ft, gt, Ht, slope)
    H64 = Ht.double().cpu().numpy()
    ref = oracle.gat(S.row_ptr, S.col_idx, vals, f, g, H64, heads, slope)
    mag = oracle.gat(S.row_ptr, S.col_idx, vals, f, g, np.abs(H64), heads, slope)
    rows = np.repeat(np.arange(S.m), np.diff(S.row_ptr))
    emax = float(np.max(np.abs(vals[:, None] * (f[rows] + g[S.col_idx])))) if S.nnz else 0.0
    deg = int(S.degrees().max())
    bound = 2 * (8 * emax + 2 * deg + 16) * U32 * mag + 1e-30
    got = out.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound)
    assert relF(got, ref) <= 1e-5


def test_gat_layer_and_projection():
    from paper_2203_07673_gb300 import fmm, gat
    S, rng = _graph(3, m=500)
    heads, rh, r_in = 4, 32, 48
    X = torch.from_numpy(rng.standard_normal((S.m, r_in)).astype(np.float32)).cuda()
    W = torch.from_numpy((rng.standard_normal((r_in, heads * rh)) / 8).astype(np.float32)).cuda()
    a_l = torch.from_numpy(rng.standard_normal(heads * rh).astype(np.float32)).cuda()
    a_r = torch.from_numpy(rng.standard_normal(heads * rh).astype(np.float32)).cuda()
    rp, ci = torch.from_numpy(S.row_ptr).cuda(), torch.from_numpy(S.col_idx).cuda()
    plan = fmm.Plan(rp, ci, S.n, heads * rh)
    out, H = gat.gat_layer(plan, X, W, a_l, a_r, heads)
    H64 = H.double().cpu().numpy()
    al = a_l.double().cpu().numpy().reshape(heads, rh)
    ar = a_r.double().cpu().numpy().reshape(heads, rh)
    f = np.einsum("ihk,hk->ih", H64.reshape(S.m, heads, rh), al)
    g = np.einsum("ihk,hk->ih", H64.reshape(S.n, heads, rh), ar)
    fp = fmm.gat_project(H, a_l, heads).double().cpu().numpy()
    assert relF(fp, f) <= 1e-5
    ref = oracle.gat(S.row_ptr, S.col_idx, None, fp, fmm.gat_project(H, a_r, heads).double()
                     .cpu().numpy(), H64, heads, 0.2)
    assert relF(out.double().cpu().numpy(), ref) <= 1e-5


def test_gat_empty_rows_and_no_edges():
    from paper_2203_07673_gb300 import fmm
    rp = torch.zeros(9, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    plan = fmm.Plan(rp, ci, 8, 64)
    out = torch.full((8, 64), 3.0, device="cuda")
    fmm.gat_forward(plan, 2, None, torch.zeros(8, 2, device="cuda"),
                    torch.zeros(8, 2, device="cuda"), torch.randn(8, 64, device="cuda"), out=out)
    assert not out.any()


def test_registered_values_skip_the_permutation():
    from paper_2203_07673_gb300 import fmm
    S, rng = _graph(9)
    r = 64
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B)
    plan = fmm.Plan(rp, ci, S.n, r)
    before = fmm.fusedmm_t(plan, vt, At, Bt)
    plan.set_values(vt)
    after = fmm.fusedmm_t(plan, vt, At, Bt)
    assert torch.equal(before, after)
    # a different pointer with other values is still permuted per call
    v2 = torch.from_numpy(rng.uniform(0, 1, S.nnz).astype(np.float32)).cuda()
    other = fmm.fusedmm_t(plan, v2, At, Bt)
    ref = oracle.fusedmm_t(S.row_ptr, S.col_idx, v2.cpu().numpy(), A, B, S.n)
    assert relF(other.double().cpu().numpy(), ref) <= 1e-5
    # changed contents must be registered again
    vt.mul_(2.0)
    plan.set_values(vt)
    doubled = fmm.fusedmm_t(plan, vt, At, Bt)
    assert relF(doubled.double().cpu().numpy(), 2 * before.double().cpu().numpy()) <= 1e-6
    dA, dB, ds = fmm.fusedmm_bwd(plan, vt, At, Bt, torch.ones(S.m, r, device="cuda"))
    e = oracle.fusedmm_grad(S.row_ptr, S.col_idx, 2 * vals.astype(np.float64), A, B,
                            np.ones((S.m, r)), S.n)
    assert relF(dB.double().cpu().numpy(), e[1]) <= 1e-5
    plan.set_values(None)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("offset_bytes", [16, 32], ids=["16B", "32B"])
def test_gat_h_alignment(offset_bytes, dtype):
    """H rows are loaded 32 bytes at a time: H that is only 16-byte aligned
    takes the generic kernel (float32) or the 8-per-lane shape with 16-byte
    loads (bfloat16); every path must match the oracle."""
    from paper_2203_07673_gb300 import fmm
    S, rng = _graph(21, m=400)
    heads, rh = 4, 32
    r = heads * rh
    H = (rng.standard_normal((S.n, r)) * 0.5).astype(np.float32)
    f = rng.standard_normal((S.m, heads)).astype(np.float32)
    g = rng.standard_normal((S.n, heads)).astype(np.float32)
    esz = torch.tensor([], dtype=dtype).element_size()
    offset = offset_bytes // esz
    buf = torch.zeros(S.n * r + 64 // esz, device="cuda", dtype=dtype)
    Hd = torch.from_numpy(H).to(dtype)
    buf[offset:offset + S.n * r] = Hd.reshape(-1).cuda()
    Ht = buf[offset:offset + S.n * r].view(S.n, r)
    assert (Ht.data_ptr() % 32 == 0) == (offset_bytes == 32)
    rp, ci = torch.from_numpy(S.row_ptr).cuda(), torch.from_numpy(S.col_idx).cuda()
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=256)
    out = fmm.gat_forward(plan, heads, None, torch.from_numpy(f).cuda(),
                          torch.from_numpy(g).cuda(), Ht, 0.2)
    ref = oracle.gat(S.row_ptr, S.col_idx, None, f, g, Hd.double().numpy(), heads, 0.2)
    assert relF(out.double().cpu().numpy(), ref) <= 1e-5
