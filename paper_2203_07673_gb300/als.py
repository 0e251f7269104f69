"""Alternating least squares with batched conjugate gradients (Sec. VI-E).

Collaborative filtering fits C ~ A B^T on the observed entries c_ij (the
nonzeros of S) by minimising sum (c_ij - <A_i, B_j>)^2 + lam (|A|^2 + |B|^2).
With B fixed each row A_i solves (sum_j B_j B_j^T + lam I) A_i = sum_j c_ij B_j
and vice versa.  As in the paper, CG solves all rows at once: every CG query
M p is one FusedMM over the 0/1 pattern (FusedMMA for the A side, FusedMMB for
the B side), the right-hand sides are one SpMM of the observations, and the
per-row vector work of each CG step is one kernel (fmm_cg_update).  All of it
runs in libfmm's kernels; this module only sequences the calls and owns the
float32 work vectors (allocated once per solver).
"""
from __future__ import annotations

import torch

from . import fmm


class ALS:
    """ALS on one pattern.  ``plan`` must be float32 with S^T; ``c`` holds the
    observations (nnz float32, CSR order); A (m x r) and B (n x r) are
    float32 and are updated in place."""

    def __init__(self, plan: fmm.Plan, c: torch.Tensor, A: torch.Tensor, B: torch.Tensor,
                 lam: float):
        if plan.dtype != torch.float32:
            raise TypeError("ALS needs a float32 plan")
        self.plan, self.c, self.A, self.B, self.lam = plan, c, A, B, float(lam)
        dev, r = plan.device, plan.r
        rows = max(plan.m, plan.n)
        self._work = [torch.empty(rows, r, device=dev) for _ in range(4)]
        self._rs = torch.empty(rows, device=dev)

    def _side(self, side: int, iters: int):
        p_, m, n = self.plan, self.plan.m, self.plan.n
        rows = m if side == 0 else n
        X = self.A if side == 0 else self.B
        b, res, p, q = (w[:rows] for w in self._work)
        rs = self._rs[:rows]
        if side == 0:
            fmm.spmm(p_, self.c, self.B, out=b)
            fmm.fusedmm(p_, None, self.A, self.B, out=q)
        else:
            fmm.spmm_t(p_, self.c, self.A, out=b)
            fmm.fusedmm_t(p_, None, self.A, self.B, out=q)
        fmm.cg_init(self.lam, b, q, X, res, p, rs)
        for _ in range(iters):
            if side == 0:
                fmm.fusedmm(p_, None, p, self.B, out=q)
            else:
                fmm.fusedmm_t(p_, None, self.A, p, out=q)
            fmm.cg_update(self.lam, X, res, p, q, rs)

    def update_a(self, iters: int = 10):
        self._side(0, iters)

    def update_b(self, iters: int = 10):
        self._side(1, iters)

    def sweep(self, iters: int = 10):
        """One ALS sweep as benchmarked in the paper: `iters` CG iterations
        for A, then `iters` for B."""
        self.update_a(iters)
        self.update_b(iters)

    def loss(self) -> float:
        """sum (c - <A_i, B_j>)^2 + lam (|A|^2 + |B|^2) (SDDMM of the pattern)."""
        pred = fmm.sddmm(self.plan, None, self.A, self.B)
        return float(((self.c - pred) ** 2).sum() + self.lam * ((self.A ** 2).sum()
                                                               + (self.B ** 2).sum()))
