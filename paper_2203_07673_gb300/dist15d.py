"""Distributed FusedMM (Sec. V), replication factor c = 1: the 1.5D
dense-shifting algorithm with local kernel fusion (Algorithm 1,
FusedMM15D) and the 1.5D sparse-shifting algorithm (SparseShift15D).

p ranks in one ring (a p x 1 grid: replication factor c = 1).  Rank k owns
  * a block of rows of S (R_k, balanced by nonzeros), the same rows of A and of
    the FusedMMA output,
  * one block of columns of S = rows of B (C_k, n / p rows each) and the same
    rows of the FusedMMB output.
Its rows of S are cut by column block into p local patterns S_{k,l}, each with
its own plan.  A FusedMMA runs p phases: in phase t rank k holds B block
l = (k + t) mod p, adds FusedMMA(S_{k,l}, A_k, B_l) to its output rows
(local kernel fusion: the SDDMM values stay in registers, one round of shifts
serves both halves, Sec. V "Local Kernel Fusion") and passes B_l to rank
k - 1 while the next block arrives from k + 1; the shift of the next block is
posted before the phase's kernel, so it overlaps it.  FusedMMB and the B
gradient follow Algorithm 1's SpMMB mode: the output block travels with its B
block, every rank adds its contribution, and after p phases and p shifts the
block is back at its owner.  The A gradient stays local (like FusedMMA), ds
is per nonzero.

This module holds index arithmetic and the schedule only.  The local work is
done by `ops` (default: the library's kernels through fmm: plans over
S_{k,l}, fmm_fusedmm_acc, fmm_fusedmm_t_acc, fmm_fusedmm_bwd_acc); the
shifts by torch.distributed point-to-point calls (NCCL moves device tensors;
with gloo the blocks are staged through host memory).  No kernel is handed
another rank's memory.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def row_bounds_by_nnz(row_ptr, parts: int) -> np.ndarray:
    """Row block boundaries (parts + 1 entries) splitting the rows of a CSR
    into `parts` consecutive blocks of about nnz / parts nonzeros each."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    m = rp.shape[0] - 1
    nnz = int(rp[-1])
    targets = [(k * nnz) // parts for k in range(parts + 1)]
    bounds = np.searchsorted(rp, targets, side="left").astype(np.int64)
    bounds[0], bounds[-1] = 0, m
    return bounds


def col_bounds_uniform(n: int, parts: int) -> np.ndarray:
    """Column block boundaries (parts + 1 entries): blocks of n / parts."""
    return np.array([(l * n) // parts for l in range(parts + 1)], dtype=np.int64)


def split_by_column_blocks(row_ptr: torch.Tensor, col_idx: torch.Tensor, col_bounds):
    """The local pattern of each column block of a row block's CSR.

    row_ptr (rows + 1) and col_idx (nnz) are int32 tensors with global column
    indices.  Returns a list with one entry per block l:
    (row_ptr_l int32, col_idx_l int32 (columns relative to the block start),
    slots_l int64: the position in the input CSR of each nonzero of S_l)."""
    dev = col_idx.device
    rows = row_ptr.numel() - 1
    nnz = col_idx.numel()
    deg = (row_ptr[1:] - row_ptr[:-1]).long()
    row_of = torch.repeat_interleave(torch.arange(rows, device=dev), deg)
    cb = torch.as_tensor(np.asarray(col_bounds, dtype=np.int64), device=dev)
    block = torch.searchsorted(cb, col_idx.long(), right=True) - 1
    # stable order by (block, row); within a row the input order is kept
    key = block * (rows + 1) + row_of
    order = torch.sort(key, stable=True).indices
    out = []
    counts = torch.bincount(block, minlength=len(col_bounds) - 1).tolist()
    start = 0
    for l, c in enumerate(counts):
        sel = order[start:start + c]
        start += c
        rp = torch.zeros(rows + 1, dtype=torch.int64, device=dev)
        if c:
            rp[1:] = torch.cumsum(torch.bincount(row_of[sel], minlength=rows), 0)
        ci = (col_idx[sel].long() - int(col_bounds[l])).to(torch.int32)
        out.append((rp.to(torch.int32), ci, sel))
    assert start == nnz
    return out


class LibraryOps:
    """Local kernels of the library (fmm): one plan per local pattern."""

    def __init__(self):
        from . import fmm
        self.fmm = fmm

    def plan(self, row_ptr, col_idx, n, r, dtype):
        return self.fmm.Plan(row_ptr, col_idx, n, r, dtype)

    def fusedmm(self, plan, vals, A, B, out):
        self.fmm.fusedmm(plan, vals, A, B, out=out)

    def fusedmm_t(self, plan, vals, A, B, out):
        self.fmm.fusedmm_t(plan, vals, A, B, out=out)

    def fusedmm_bwd(self, plan, vals, A, B, G, dA, dB, ds):
        self.fmm.fusedmm_bwd(plan, vals, A, B, G, out=(dA, dB, ds))

    def fusedmm_acc(self, plan, vals, A, B, out):
        self.fmm.fusedmm_acc(plan, vals, A, B, out)

    def fusedmm_t_acc(self, plan, vals, A, B, out):
        self.fmm.fusedmm_t_acc(plan, vals, A, B, out)

    def fusedmm_bwd_acc(self, plan, vals, A, B, G, dA, dB, ds):
        self.fmm.fusedmm_bwd_acc(plan, vals, A, B, G, dA, dB, ds)

    def sddmm_acc(self, plan, vals, A, B, v):
        self.fmm.sddmm_acc(plan, vals, A, B, v)

    def spmm(self, plan, v, B, out):
        self.fmm.spmm(plan, v, B, out=out)

    def spmm_t_acc(self, plan, v, A, out):
        self.fmm.spmm_t_acc(plan, v, A, out)

    def close(self, plan):
        plan.close()


class FusedMM15D:
    """FusedMMA, FusedMMB and the FusedMMA adjoint of one distributed S.

    Every rank of `group` calls every method with its own blocks:
      row_ptr, col_idx  its rows of S (int32, global column indices)
      n, r, dtype       global columns of S, dense width, dense dtype
      col_bounds        column block boundaries (default: n / p each)
    A_k is (rows, r) and B_k (cols of block k, r), both of `dtype`; vals_k
    (nnz of the rank's rows, float32, rank-local CSR order) or None (all
    ones).  Outputs are float32."""

    def __init__(self, row_ptr, col_idx, n, r, dtype=torch.float32, group=None, col_bounds=None,
                 ops=None):
        self.group = group
        # without a process group: one rank (p = 1, no shifts)
        self.p = dist.get_world_size(group) if dist.is_initialized() else 1
        self.k = dist.get_rank(group) if dist.is_initialized() else 0
        self.n, self.r, self.dtype = int(n), int(r), dtype
        self.col_bounds = (col_bounds_uniform(self.n, self.p) if col_bounds is None
                           else np.asarray(col_bounds, dtype=np.int64))
        self.rows = row_ptr.numel() - 1
        self.nnz = col_idx.numel()
        self.ops = ops if ops is not None else LibraryOps()
        self.blocks = split_by_column_blocks(row_ptr, col_idx, self.col_bounds)
        widths = np.diff(self.col_bounds)
        self.maxw = int(widths.max()) if len(widths) else 0
        self.plans = [self.ops.plan(rp, ci, int(widths[l]), self.r, dtype)
                      for l, (rp, ci, _) in enumerate(self.blocks)]
        # a block whose nonzeros sit consecutively in the rank's CSR takes its
        # values (and writes its ds) as a view, with no gather (always so at p = 1)
        self.spans = [self._span(sel) for _, _, sel in self.blocks]
        self.device = col_idx.device

    @staticmethod
    def _span(sel):
        c = sel.numel()
        if c == 0:
            return (0, 0)
        a = int(sel[0])
        if int(sel[-1]) - a + 1 == c and bool((sel[1:] - sel[:-1] == 1).all()):
            return (a, c)
        return None

    def close(self):
        for pl in self.plans:
            self.ops.close(pl)
        self.plans = []

    # ------------------------------------------------------------ schedule

    def block_of_phase(self, t: int) -> int:
        """The B block rank k holds in phase t."""
        return (self.k + t) % self.p

    def _width(self, l):
        return int(self.col_bounds[l + 1] - self.col_bounds[l])

    def _vals(self, vals, l):
        if vals is None:
            return None
        if self.spans[l] is not None:
            return vals.narrow(0, *self.spans[l])
        return vals.index_select(0, self.blocks[l][2])

    def _b_bufs(self, B_k):
        """The B blocks of the phases: B_k itself in phase 0 (it is only
        sent, never received into), then two receive buffers in turn.
        Shifts move maxw rows, so a narrower B_k is copied into a padded
        buffer first."""
        if B_k.shape[0] == self.maxw or self.p == 1:
            first = B_k
        else:
            first = torch.zeros((self.maxw, self.r), dtype=self.dtype, device=B_k.device)
            first[:B_k.shape[0]].copy_(B_k)
        if self.p == 1:
            return [first]
        spare = [torch.empty((self.maxw, self.r), dtype=self.dtype, device=B_k.device)
                 for _ in range(2)]
        return [first] + spare

    @staticmethod
    def _phase_buf(bufs, t):
        return bufs[0] if t == 0 else bufs[1 + (t - 1) % 2]

    def _shift(self, send, recv):
        """send -> rank k - 1, recv <- rank k + 1 (returns a waitable)."""
        dst = (self.k - 1) % self.p
        src = (self.k + 1) % self.p
        if self.p == 1:
            recv.copy_(send)
            return []
        host = dist.get_backend(self.group) == "gloo" and send.is_cuda
        if host:
            s_h, r_h = send.cpu(), torch.empty(recv.shape, dtype=recv.dtype)
            reqs = dist.batch_isend_irecv([
                dist.P2POp(dist.isend, s_h, self._global(dst), group=self.group),
                dist.P2POp(dist.irecv, r_h, self._global(src), group=self.group)])
            return [(reqs, r_h, recv)]
        reqs = dist.batch_isend_irecv([
            dist.P2POp(dist.isend, send, self._global(dst), group=self.group),
            dist.P2POp(dist.irecv, recv, self._global(src), group=self.group)])
        return [(reqs, None, None)]

    def _global(self, rank):
        return rank if self.group is None else dist.get_global_rank(self.group, rank)

    @staticmethod
    def _wait(handles):
        for reqs, r_h, recv in handles:
            for q in reqs:
                q.wait()
            if r_h is not None:
                recv.copy_(r_h)

    # ------------------------------------------------------------ operations

    def fusedmm(self, vals, A_k, B_k):
        """FusedMMA rows of this rank: out_i = sum_j s_ij <A_i, B_j> B_j."""
        out = torch.empty((self.rows, self.r), dtype=torch.float32, device=A_k.device)
        bufs = self._b_bufs(B_k)
        for t in range(self.p):
            l = self.block_of_phase(t)
            cur = self._phase_buf(bufs, t)
            # the next block is in flight while this phase computes
            pend = self._shift(cur, self._phase_buf(bufs, t + 1)) if t + 1 < self.p else []
            # phase 0 writes every output row, later phases add to them
            call = self.ops.fusedmm if t == 0 else self.ops.fusedmm_acc
            call(self.plans[l], self._vals(vals, l), A_k, cur[:self._width(l)], out)
            self._wait(pend)
        return out

    def fusedmm_t(self, vals, A_k, B_k):
        """FusedMMB rows of this rank's B block: out_j = sum_i s_ij <A_i, B_j> A_i."""
        dev = A_k.device
        bufs = self._b_bufs(B_k)
        outs = [torch.empty((self.maxw, self.r), dtype=torch.float32, device=dev)
                for _ in range(1 if self.p == 1 else 2)]
        cur = 0
        for t in range(self.p):
            l = self.block_of_phase(t)
            b = self._phase_buf(bufs, t)
            pend = self._shift(b, self._phase_buf(bufs, t + 1)) if t + 1 < self.p else []
            w = self._width(l)
            call = self.ops.fusedmm_t if t == 0 else self.ops.fusedmm_t_acc
            call(self.plans[l], self._vals(vals, l), A_k, b[:w], outs[cur][:w])
            if self.p == 1:
                break
            # the output block travels on with its B block; after p shifts it
            # is back at its owner
            self._wait(pend + self._shift(outs[cur], outs[1 - cur]))
            cur = 1 - cur
        return outs[cur][:self._width(self.k)]

    def fusedmm_bwd(self, vals, A_k, B_k, G_k):
        """Adjoint of FusedMMA for L = <G, FusedMMA>: (dA rows of this rank,
        dB rows of this rank's B block, ds of this rank's nonzeros)."""
        dev = A_k.device
        dA = torch.empty((self.rows, self.r), dtype=torch.float32, device=dev)
        ds = torch.empty(self.nnz, dtype=torch.float32, device=dev)
        bufs = self._b_bufs(B_k)
        dBs = [torch.empty((self.maxw, self.r), dtype=torch.float32, device=dev)
               for _ in range(1 if self.p == 1 else 2)]
        cur = 0
        for t in range(self.p):
            l = self.block_of_phase(t)
            b = self._phase_buf(bufs, t)
            pend = self._shift(b, self._phase_buf(bufs, t + 1)) if t + 1 < self.p else []
            w = self._width(l)
            sel, span = self.blocks[l][2], self.spans[l]
            ds_l = (ds.narrow(0, *span) if span is not None
                    else torch.empty(sel.numel(), dtype=torch.float32, device=dev))
            call = self.ops.fusedmm_bwd if t == 0 else self.ops.fusedmm_bwd_acc
            call(self.plans[l], self._vals(vals, l), A_k, b[:w], G_k, dA, dBs[cur][:w], ds_l)
            if span is None:
                ds.index_copy_(0, sel, ds_l)
            if self.p == 1:
                break
            self._wait(pend + self._shift(dBs[cur], dBs[1 - cur]))
            cur = 1 - cur
        return dA, dBs[cur][:self._width(self.k)], ds


def slice_bounds(r: int, parts: int) -> np.ndarray:
    """Column slices of the dense width r (parts + 1 boundaries)."""
    return np.array([(k * r) // parts for k in range(parts + 1)], dtype=np.int64)


class SparseShift15D:
    """FusedMMA and FusedMMB by the 1.5D sparse-shifting, dense-replicating
    algorithm (Sec. V, c = 1): the dense matrices are divided by column
    slices of r, the sparse matrix by block rows, and the block rows circulate.

    Local kernel fusion is impossible in this layout (a rank holds only a
    slice of every row of A and B, so no rank can finish a dot product before
    the aggregation, Sec. IV-B), so FusedMM runs as SDDMM then SpMM: round 1
    passes each block row's values around the ring, every rank adding its
    slice's partial dot products (fmm_sddmm_acc); after p phases and p shifts
    each block is back at its owner with its SDDMM values complete.  Round 2
    passes the completed blocks around again, every rank applying each block
    to its column slice (fmm_spmm for FusedMMA rows; fmm_spmm_t_acc, summed
    over the blocks, for FusedMMB).  The patterns are laid out on every rank
    once (one plan per block row, at the rank's slice width), so only the
    values travel: nnz/p floats per shift.

    Every rank passes the whole pattern (row_ptr, col_idx: int32 on its
    device), the values of all nonzeros (or None), its column slices A_k
    (m x r_k) and B_k (n x r_k), and gets its slices of the outputs."""

    def __init__(self, row_ptr, col_idx, n, r, dtype=torch.float32, group=None, ops=None,
                 row_bounds=None):
        self.group = group
        self.p = dist.get_world_size(group) if dist.is_initialized() else 1
        self.k = dist.get_rank(group) if dist.is_initialized() else 0
        self.n, self.r, self.dtype = int(n), int(r), dtype
        self.m = row_ptr.numel() - 1
        self.ops = ops if ops is not None else LibraryOps()
        rp_h = row_ptr.cpu().numpy()
        self.row_bounds = (row_bounds_by_nnz(rp_h, self.p) if row_bounds is None
                           else np.asarray(row_bounds, dtype=np.int64))
        self.slices = slice_bounds(self.r, self.p)
        self.width = int(self.slices[self.k + 1] - self.slices[self.k])
        self.nnz_bounds = rp_h.astype(np.int64)[self.row_bounds]
        self.plans = []
        for b in range(self.p):
            r0, r1 = int(self.row_bounds[b]), int(self.row_bounds[b + 1])
            p0, p1 = int(self.nnz_bounds[b]), int(self.nnz_bounds[b + 1])
            rp = (row_ptr[r0:r1 + 1].long() - p0).to(torch.int32)
            self.plans.append(self.ops.plan(rp, col_idx[p0:p1], self.n, self.width, dtype))
        self.maxnz = int(np.diff(self.nnz_bounds).max()) if self.p else 0
        self._ring = FusedMM15D.__new__(FusedMM15D)   # borrows its shift helpers
        self._ring.group, self._ring.p, self._ring.k = group, self.p, self.k

    def close(self):
        for pl in self.plans:
            self.ops.close(pl)
        self.plans = []

    def block_of_phase(self, t: int) -> int:
        return (self.k + t) % self.p

    def _rows(self, b):
        return int(self.row_bounds[b]), int(self.row_bounds[b + 1])

    def _nz(self, b):
        return int(self.nnz_bounds[b]), int(self.nnz_bounds[b + 1])

    def _sddmm_round(self, vals, A_k, B_k):
        """Round 1: every block row's SDDMM values, summed over the slices;
        returns (this rank's block values, padded buffer pair, current)."""
        dev = A_k.device
        bufs = [torch.zeros(self.maxnz, dtype=torch.float32, device=dev),
                torch.empty(self.maxnz, dtype=torch.float32, device=dev)]
        cur = 0
        for t in range(self.p):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            v = None if vals is None else vals[p0:p1]
            self.ops.sddmm_acc(self.plans[b], v, A_k[r0:r1], B_k, bufs[cur][:p1 - p0])
            self._ring._wait(self._ring._shift(bufs[cur], bufs[1 - cur]))
            cur = 1 - cur
        return bufs, cur

    def fusedmm(self, vals, A_k, B_k):
        """This rank's column slice of FusedMMA (m x r_k)."""
        bufs, cur = self._sddmm_round(vals, A_k, B_k)
        out = torch.empty((self.m, self.width), dtype=torch.float32, device=A_k.device)
        for t in range(self.p):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            pend = self._ring._shift(bufs[cur], bufs[1 - cur]) if t + 1 < self.p else []
            self.ops.spmm(self.plans[b], bufs[cur][:p1 - p0], B_k, out[r0:r1])
            self._ring._wait(pend)
            cur = 1 - cur
        return out

    def fusedmm_t(self, vals, A_k, B_k):
        """This rank's column slice of FusedMMB (n x r_k)."""
        bufs, cur = self._sddmm_round(vals, A_k, B_k)
        out = torch.zeros((self.n, self.width), dtype=torch.float32, device=A_k.device)
        for t in range(self.p):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            pend = self._ring._shift(bufs[cur], bufs[1 - cur]) if t + 1 < self.p else []
            self.ops.spmm_t_acc(self.plans[b], bufs[cur][:p1 - p0], A_k[r0:r1], out)
            self._ring._wait(pend)
            cur = 1 - cur
        return out
