"""ALS with batched CG (Sec. VI-E) on the GPU against the FP64 oracle.

Tolerance: the GPU runs CG in float32.  Each CG query M p carries a relative
rounding error of at most about (r + deg + 4) u (u = 2^-24, the FusedMM
bound of the parity tests) and each row update a few u; CG on these
well-conditioned systems (lambda = 1) does not amplify them much over a few
iterations, so k iterations are compared with a relative Frobenius bound of
k (r + deg_max + 4) u times a conditioning allowance of 100.
"""
import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, deg_max, relF
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem(seed, m=600, n=450, r=64):
    rng = np.random.default_rng(seed)
    S = wl.random_csr(m, n, rng, mean_deg=12, empty_frac=0.05, hubs=((3, 400),))
    c = wl.half_steps(S.nnz, 1.0, 5.0, rng)
    A = (rng.standard_normal((m, r)) * 0.3).astype(np.float32)
    B = (rng.standard_normal((n, r)) * 0.3).astype(np.float32)
    return S, c, A, B


def test_cg_update_kernel_one_step():
    from paper_2203_07673_gb300 import fmm
    rng = np.random.default_rng(0)
    for rows, r in ((300, 64), (257, 100), (64, 300)):
        x, res, p, q = (rng.standard_normal((rows, r)).astype(np.float32) for _ in range(4))
        rs = (res.astype(np.float64) ** 2).sum(1).astype(np.float32)
        lam = 0.7
        T = [torch.from_numpy(a.copy()).cuda() for a in (x, res, p, q)]
        rs_t = torch.from_numpy(rs.copy()).cuda()
        fmm.cg_update(lam, T[0], T[1], T[2], T[3], rs_t)
        # the definition in float64
        x64, r64, p64, q64 = (a.astype(np.float64) for a in (x, res, p, q))
        t = q64 + lam * p64
        pq = (p64 * t).sum(1)
        alpha = np.where(pq > 0, rs / pq, 0.0)[:, None]
        x64 += alpha * p64
        r64 -= alpha * t
        rs2 = (r64 ** 2).sum(1)
        beta = np.where(rs > 0, rs2 / rs, 0.0)[:, None]
        p64 = r64 + beta * p64
        for name, got, exp in (("x", T[0], x64), ("res", T[1], r64), ("p", T[2], p64),
                               ("rs", rs_t, rs2)):
            assert relF(got.double().cpu().numpy(), exp) <= 1e-5, name


@pytest.mark.parametrize("r", [32, 64, 100])
def test_als_cg_matches_oracle(r):
    from paper_2203_07673_gb300 import als, fmm
    S, c, A, B = _problem(r, r=r)
    lam, iters = 1.0, 5
    rp, ci = torch.from_numpy(S.row_ptr).cuda(), torch.from_numpy(S.col_idx).cuda()
    plan = fmm.Plan(rp, ci, S.n, r)
    At, Bt = torch.from_numpy(A.copy()).cuda(), torch.from_numpy(B.copy()).cuda()
    solver = als.ALS(plan, torch.from_numpy(c).cuda(), At, Bt, lam)
    bound = iters * (r + deg_max(S) + 4) * U32 * 100
    solver.update_a(iters)
    A1 = oracle.als_cg(S.row_ptr, S.col_idx, c, A, B, lam, iters, 0)
    assert relF(At.double().cpu().numpy(), A1) <= bound
    solver.update_b(iters)
    # the B update starts from the GPU's A, as the solver does
    B1 = oracle.als_cg(S.row_ptr, S.col_idx, c, At.double().cpu().numpy(), B, lam, iters, 1)
    assert relF(Bt.double().cpu().numpy(), B1) <= bound


def test_als_loss_decreases_on_gpu():
    from paper_2203_07673_gb300 import als, fmm
    S, c, A, B = _problem(7, r=32)
    rp, ci = torch.from_numpy(S.row_ptr).cuda(), torch.from_numpy(S.col_idx).cuda()
    plan = fmm.Plan(rp, ci, S.n, 32)
    solver = als.ALS(plan, torch.from_numpy(c).cuda(), torch.from_numpy(A).cuda(),
                     torch.from_numpy(B).cuda(), 0.5)
    prev = solver.loss()
    for _ in range(3):
        solver.sweep(10)
        cur = solver.loss()
        assert cur <= prev * (1 + 1e-5)
        prev = cur
