"""FusedMM as a torch.autograd.Function: gradients against the FP64 oracle.

The oracle's gradients are themselves pinned to central finite differences
and to dense closed forms (tests/test_oracle_pins.py).  bfloat16 inputs get
bfloat16 gradients (float32 results rounded once), so those are compared
with one extra bfloat16 rounding (2^-8 relative) on top of the float32 bound.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, deg_max, relF, upload
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _check(name, got, ref, mag, terms, bf16):
    got = got.detach().double().cpu().numpy()
    bound = 2.0 * terms * U32 * mag + 1e-30
    if bf16:
        bound = bound + 2.0 ** -8 * np.abs(ref)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{name}: {bad.sum()} elements over the bound"
    assert relF(got, ref) <= (2e-2 if bf16 else 1e-5), name


@pytest.mark.parametrize("transpose", [False, True], ids=["A", "B"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [64, 128, 20])
def test_autograd_gradients(r, dtype, transpose):
    from paper_2203_07673_gb300 import autograd, fmm
    rng = np.random.default_rng(r + 7 * transpose)
    S = wl.random_csr(400, 300, rng, mean_deg=6, empty_frac=0.1, dup_frac=0.1,
                      hubs=((9, 900),))
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    A = (rng.standard_normal((S.m, r)) / np.sqrt(r)).astype(np.float32)
    B = (rng.standard_normal((S.n, r)) / np.sqrt(r)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
    vt.requires_grad_(True); At.requires_grad_(True); Bt.requires_grad_(True)
    plan = fmm.Plan(rp, ci, S.n, r, dtype, split_nnz=128)
    out = autograd.fusedmm(plan, vt, At, Bt, transpose=transpose)
    G = torch.randn(out.shape, device="cuda")
    out.backward(G)
    assert At.grad.dtype == dtype and Bt.grad.dtype == dtype and vt.grad.dtype == torch.float32
    A64 = At.detach().double().cpu().numpy()
    B64 = Bt.detach().double().cpu().numpy()
    G64 = G.double().cpu().numpy()
    grad = oracle.fusedmm_t_grad if transpose else oracle.fusedmm_grad
    fwd = oracle.fusedmm_t if transpose else oracle.fusedmm
    ref = grad(S.row_ptr, S.col_idx, vals, A64, B64, G64, S.n)
    mag = grad(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), np.abs(G64), S.n)
    terms = 2 * r + deg_max(S) + 4
    bf16 = dtype == torch.bfloat16
    _check("out", out, fwd(S.row_ptr, S.col_idx, vals, A64, B64, S.n),
           fwd(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n), terms, False)
    _check("dA", At.grad, ref[0], mag[0], terms, bf16)
    _check("dB", Bt.grad, ref[1], mag[1], terms, bf16)
    _check("ds", vt.grad, ref[2], mag[2], terms, False)


def test_autograd_partial_requirements():
    # only B requires a gradient: the others are skipped
    from paper_2203_07673_gb300 import autograd, fmm
    rng = np.random.default_rng(3)
    S = wl.random_csr(100, 80, rng, mean_deg=4)
    A = rng.standard_normal((100, 32)).astype(np.float32)
    B = rng.standard_normal((80, 32)).astype(np.float32)
    rp, ci, _, At, Bt = upload(S, None, A, B)
    Bt.requires_grad_(True)
    plan = fmm.Plan(rp, ci, S.n, 32)
    out = autograd.fusedmm(plan, None, At, Bt)
    out.sum().backward()
    assert At.grad is None and Bt.grad is not None
    ref = oracle.fusedmm_grad(S.row_ptr, S.col_idx, None, A, B, np.ones((100, 32)), S.n)[1]
    assert relF(Bt.grad.double().cpu().numpy(), ref) <= 1e-5
