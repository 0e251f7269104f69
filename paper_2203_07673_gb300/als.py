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

    def start(self, side: int):
        """CG set-up of one side (0: rows of A, 1: rows of B): b = SpMM of the
        observations, q = the FusedMM of the current rows, then
        res = b - q - lam x, p = res, rs = <res, res> (fmm_cg_init)."""
        p_, rows = self.plan, self._rows(side)
        X = self.A if side == 0 else self.B
        b, res, p, q = (w[:rows] for w in self._work)
        if side == 0:
            fmm.spmm(p_, self.c, self.B, out=b)
            fmm.fusedmm(p_, None, self.A, self.B, out=q)
        else:
            fmm.spmm_t(p_, self.c, self.A, out=b)
            fmm.fusedmm_t(p_, None, self.A, self.B, out=q)
        fmm.cg_init(self.lam, b, q, X, res, p, self._rs[:rows])

    def iterate(self, side: int, iters: int):
        """`iters` CG iterations of one side from the state left by start()
        or an earlier iterate(): q = the FusedMM of p, then fmm_cg_update."""
        p_, rows = self.plan, self._rows(side)
        X = self.A if side == 0 else self.B
        _, res, p, q = (w[:rows] for w in self._work)
        rs = self._rs[:rows]
        for _ in range(iters):
            if side == 0:
                fmm.fusedmm(p_, None, p, self.B, out=q)
            else:
                fmm.fusedmm_t(p_, None, self.A, p, out=q)
            fmm.cg_update(self.lam, X, res, p, q, rs)

    def state(self, side: int):
        """Views of the CG state of a side: (res, p, rs)."""
        rows = self._rows(side)
        return self._work[1][:rows], self._work[2][:rows], self._rs[:rows]

    def _rows(self, side: int) -> int:
        return self.plan.m if side == 0 else self.plan.n

    def _side(self, side: int, iters: int):
        self.start(side)
        self.iterate(side, iters)

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
