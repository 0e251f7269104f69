"""Distributed FusedMM (Sec. V) on a (p/c) x c grid of ranks: the 1.5D
dense-shifting, dense-replicating algorithm with local kernel fusion
(Algorithm 1, FusedMM15D), the same grid with replication reuse instead of
local kernel fusion (Sec. IV-B strategy (1), ReplicationReuse15D), and the
1.5D sparse-shifting, dense-replicating algorithm (SparseShift15D).

The grid (Sec. V, "1.5D Dense Shifting, Dense Replicating"): p ranks form c
layers of p/c ranks each; rank k sits in layer k // (p/c) at position
q = k % (p/c).  The c ranks of one position q, one per layer, form a fiber.
Dense matrices are cut into p row blocks (A and the FusedMMA output by rows
of S, balanced by nonzeros; B and the FusedMMB output by columns of S,
n / p each).  Within a layer, dense blocks travel around a ring (each shift
sends to position q - 1 and receives from q + 1; the shift of the next
block is posted before a phase's kernel, so it overlaps it); along a fiber,
the replicated matrix is all-gathered once and a replicated output is
reduce-scattered once.  With c = 1 there is one layer, no fiber
communication, and the grid is the ring of p ranks.

FusedMM15D (local kernel fusion, A replicated, B shifting):
  * rank (q, l) owns A block q c + l (and its rows of the FusedMMA output,
    dA) and B block l (p/c) + q (and its rows of the FusedMMB output, dB);
  * its local S is S[T_q, C_l]: the rows T_q of the fiber's c A blocks and
    the columns C_l of the layer's p/c B blocks, cut by B block into p/c
    local patterns, each with its own plan;
  * FusedMMA: all-gather A over the fiber into T (rows T_q), then p/c phases
    out_T += FusedMMA(S[T_q, block], T, B_block) while B shifts around the
    layer (the SDDMM values stay in registers: one round of shifts serves
    both halves), then reduce-scatter out_T over the fiber;
  * FusedMMB and dB: the output block travels with its B block (Algorithm
    1's SpMMB mode); after p/c phases and p/c shifts it is back at its
    owner, complete (every layer covers all rows of S);
  * dA like FusedMMA (reduce-scattered), ds per local nonzero.

ReplicationReuse15D (no local kernel fusion, B replicated, A shifting):
FusedMMA as an SDDMM round and an SpMM round that both use the B rows
replicated once along the fiber; the output is the travelling matrix, so no
reduce-scatter is needed: one all-gather and 2 p/c shifts (Sec. V,
"Communication analysis, Replication Reuse").
  * rank (q, l) owns A block l (p/c) + q (and its output rows) and B block
    q c + l; its local S is S[R_l, C_q]: the rows of the layer's p/c A
    blocks and the columns of the fiber's c B blocks, cut by A block;
  * round 1: A blocks travel around the layer; the rank computes the SDDMM
    values of its piece for each block it holds (they stay with the rank);
  * round 2: the output blocks travel; the rank adds SpMM(piece, values,
    replicated B rows) to each block it holds; after p/c shifts each block is
    back at its owner.

This module holds index arithmetic and the schedule only.  The local work is
done by `ops` (default: the library's kernels through fmm); the shifts and
fiber collectives by torch.distributed (NCCL moves device tensors; with
gloo the blocks are staged through host memory).  No kernel is handed
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


def local_block(row_ptr, col_idx, r0: int, r1: int, c0: int, c1: int):
    """The part of a CSR in rows [r0, r1) and columns [c0, c1): (row_ptr
    int32 (r1 - r0 + 1), col_idx int32 (global columns), slots int64: the
    position of each of its nonzeros in the input CSR), in the input order.
    Works on host or device tensors (int32)."""
    dev = col_idx.device
    p0, p1 = int(row_ptr[r0]), int(row_ptr[r1])
    ci = col_idx[p0:p1].long()
    keep = (ci >= c0) & (ci < c1)
    deg = (row_ptr[r0 + 1:r1 + 1] - row_ptr[r0:r1]).long()
    row_of = torch.repeat_interleave(torch.arange(r1 - r0, device=dev), deg)
    counts = torch.bincount(row_of[keep], minlength=r1 - r0)
    rp = torch.zeros(r1 - r0 + 1, dtype=torch.int64, device=dev)
    rp[1:] = torch.cumsum(counts, 0)
    slots = torch.nonzero(keep).flatten() + p0
    return rp.to(torch.int32), ci[keep].to(torch.int32), slots


def split_by_column_blocks(row_ptr: torch.Tensor, col_idx: torch.Tensor, col_bounds):
    """The local pattern of each column block of a row block's CSR.

    row_ptr (rows + 1) and col_idx (nnz) are int32 tensors with global column
    indices, all inside [col_bounds[0], col_bounds[-1]).  Returns a list with
    one entry per block l: (row_ptr_l int32, col_idx_l int32 (columns
    relative to the block start), slots_l int64: the position in the input
    CSR of each nonzero of S_l)."""
    dev = col_idx.device
    rows = row_ptr.numel() - 1
    nnz = col_idx.numel()
    if nnz and (int(col_idx.min()) < int(col_bounds[0]) or int(col_idx.max()) >= int(col_bounds[-1])):
        raise ValueError("split_by_column_blocks: a column lies outside the column blocks")
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


def _span(sel):
    """(first, count) when the slots are consecutive, else None."""
    c = sel.numel()
    if c == 0:
        return (0, 0)
    a = int(sel[0])
    if int(sel[-1]) - a + 1 == c and bool((sel[1:] - sel[:-1] == 1).all()):
        return (a, c)
    return None


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

    def sddmm(self, plan, vals, A, B, v):
        self.fmm.sddmm(plan, vals, A, B, out=v)

    def sddmm_acc(self, plan, vals, A, B, v):
        self.fmm.sddmm_acc(plan, vals, A, B, v)

    def spmm(self, plan, v, B, out):
        self.fmm.spmm(plan, v, B, out=out)

    def spmm_acc(self, plan, v, B, out):
        self.fmm.spmm_acc(plan, v, B, out)

    def spmm_t_acc(self, plan, v, A, out):
        self.fmm.spmm_t_acc(plan, v, A, out)

    def close(self, plan):
        plan.close()


class Grid15D:
    """The (p/c) x c grid over the ranks of `group` (the default group when
    c > 1: the fiber groups are created by every rank).  Without a process
    group: p = 1."""

    def __init__(self, c: int = 1, group=None):
        self.group = group
        self.p = dist.get_world_size(group) if dist.is_initialized() else 1
        self.k = dist.get_rank(group) if dist.is_initialized() else 0
        c = int(c)
        if c < 1 or self.p % c:
            raise ValueError(f"replication factor {c} must divide the {self.p} ranks")
        if c > 1 and group is not None:
            raise ValueError("replication factor > 1 needs the default process group")
        self.c = c
        self.lp = self.p // c                     # ranks per layer
        self.layer, self.q = divmod(self.k, self.lp)
        self.fiber_group = None
        if self.p > 1 and c > 1:
            # every rank creates every fiber group, in the same order
            for q in range(self.lp):
                g = dist.new_group([l * self.lp + q for l in range(c)])
                if q == self.q:
                    self.fiber_group = g
        self.gloo = self.p > 1 and dist.get_backend(group) == "gloo"

    def rank_of(self, q: int, layer: int) -> int:
        """Global rank of position q in `layer`."""
        r = layer * self.lp + q
        return r if self.group is None else dist.get_global_rank(self.group, r)

    # ------------------------------------------------------------ transfers

    def shift(self, send, recv):
        """Layer ring: send -> position q - 1, recv <- q + 1 (returns a
        waitable list; with one rank per layer, recv = send)."""
        if self.lp == 1:
            recv.copy_(send)
            return []
        dst = self.rank_of((self.q - 1) % self.lp, self.layer)
        src = self.rank_of((self.q + 1) % self.lp, self.layer)
        if self.gloo and (send.is_cuda or send.dtype == torch.bfloat16):
            # staged through host memory, as raw bytes (gloo moves no bfloat16)
            s_h = _as_bytes(send.cpu())
            r_h = torch.empty(s_h.shape, dtype=torch.uint8)
            reqs = dist.batch_isend_irecv([
                dist.P2POp(dist.isend, s_h, dst, group=self.group),
                dist.P2POp(dist.irecv, r_h, src, group=self.group)])
            return [(reqs, r_h, recv)]
        reqs = dist.batch_isend_irecv([
            dist.P2POp(dist.isend, send, dst, group=self.group),
            dist.P2POp(dist.irecv, recv, src, group=self.group)])
        return [(reqs, None, None)]

    @staticmethod
    def wait(handles):
        for reqs, r_h, recv in handles:
            for q in reqs:
                q.wait()
            if r_h is not None:
                recv.copy_(r_h.view(recv.dtype).view(recv.shape))

    def gather_fiber(self, X, counts):
        """All-gather along the fiber: the rows of the c blocks (block l of
        counts[l] rows held by the fiber's rank in layer l), concatenated in
        layer order."""
        if self.c == 1:
            return X
        mx = max(int(x) for x in counts)
        buf = torch.zeros((mx,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
        buf[:X.shape[0]].copy_(X)
        host = self.gloo and X.is_cuda
        src = buf.cpu() if host else buf
        raw = self.gloo and X.dtype == torch.bfloat16
        if raw:
            src = _as_bytes(src)                  # gloo moves no bfloat16: raw bytes
        parts = [torch.empty_like(src) for _ in range(self.c)]
        dist.all_gather(parts, src, group=self.fiber_group)
        if raw:
            parts = [q.view(X.dtype).view(buf.shape) for q in parts]
        T = torch.cat([parts[l][:int(counts[l])] for l in range(self.c)])
        return T.to(X.device)

    def reduce_scatter_fiber(self, T, offs):
        """Sum over the fiber of T (rows offs[0]..offs[c], float32); the rank
        in layer l keeps rows [offs[l], offs[l + 1]) of the sum."""
        if self.c == 1:
            return T
        host = self.gloo and T.is_cuda
        src = T.cpu() if host else T
        mine = None
        for l in range(self.c):
            blk = src[int(offs[l]):int(offs[l + 1])].clone()
            dist.reduce(blk, dst=self.rank_of(self.q, l), group=self.fiber_group)
            if l == self.layer:
                mine = blk
        return mine.to(T.device)


def _as_bytes(t):
    """A contiguous tensor's bytes as a flat uint8 tensor (same storage)."""
    return t.contiguous().view(-1).view(torch.uint8)


def _phase_buf(bufs, t):
    """Phase t's block: the rank's own block in phase 0 (only ever sent),
    then two receive buffers in turn."""
    return bufs[0] if t == 0 else bufs[1 + (t - 1) % 2]


def _travel_bufs(X, rows, r, dtype, lp):
    """Buffers of a travelling dense block: X itself for phase 0 (padded to
    `rows` when narrower: every shift moves `rows` rows), then two spares."""
    if X.shape[0] == rows or lp == 1:
        first = X
    else:
        first = torch.zeros((rows, r), dtype=dtype, device=X.device)
        first[:X.shape[0]].copy_(X)
    if lp == 1:
        return [first]
    return [first] + [torch.empty((rows, r), dtype=dtype, device=X.device) for _ in range(2)]


class FusedMM15D:
    """FusedMMA, FusedMMB and the FusedMMA adjoint of one distributed S by
    Algorithm 1 with local kernel fusion, replication factor c.

    Every rank of the grid calls every method with its own blocks:
      row_ptr, col_idx  its local S = S[T_q, C_l] (int32, global column
                        indices): the rows of its fiber's c A blocks and the
                        columns of its layer's p/c B blocks
      n, r, dtype       global columns of S, dense width, dense dtype
      col_bounds        B block boundaries, p + 1 (default: n / p each)
      row_bounds        A block boundaries, p + 1 (needed when c > 1)
    A_k (rows of A block q c + l, r) and B_k (rows of B block l p/c + q, r),
    both of `dtype`; vals_k (nnz of the local S, float32, local CSR order)
    or None (all ones).  Outputs are float32."""

    def __init__(self, row_ptr, col_idx, n, r, dtype=torch.float32, group=None, col_bounds=None,
                 ops=None, c=1, row_bounds=None):
        self.grid = Grid15D(c, group)
        g = self.grid
        self.p, self.k, self.c, self.lp = g.p, g.k, g.c, g.lp
        self.n, self.r, self.dtype = int(n), int(r), dtype
        self.col_bounds = (col_bounds_uniform(self.n, self.p) if col_bounds is None
                           else np.asarray(col_bounds, dtype=np.int64))
        self.rows = row_ptr.numel() - 1
        self.nnz = col_idx.numel()
        if self.c > 1:
            if row_bounds is None:
                raise ValueError("row_bounds (A block boundaries) are needed when c > 1")
            rb = np.asarray(row_bounds, dtype=np.int64)
            counts = np.diff(rb[g.q * self.c:(g.q + 1) * self.c + 1])
            if int(counts.sum()) != self.rows:
                raise ValueError("the local S must hold the rows of the fiber's A blocks")
        else:
            counts = np.array([self.rows], dtype=np.int64)
        self.fiber_counts = counts
        self.t_offs = np.concatenate([[0], np.cumsum(counts)])
        self.ops = ops if ops is not None else LibraryOps()
        lb = self.col_bounds[g.layer * self.lp:(g.layer + 1) * self.lp + 1]
        self.blocks = split_by_column_blocks(row_ptr, col_idx, lb)
        self.widths = np.diff(lb)
        self.maxw = int(self.widths.max()) if len(self.widths) else 0
        self.plans = [self.ops.plan(rp, ci, int(self.widths[l]), self.r, dtype)
                      for l, (rp, ci, _) in enumerate(self.blocks)]
        # a block whose nonzeros sit consecutively in the local CSR takes its
        # values (and writes its ds) as a view, with no gather (always so
        # with one rank per layer)
        self.spans = [_span(sel) for _, _, sel in self.blocks]
        self.device = col_idx.device

    def close(self):
        for pl in self.plans:
            self.ops.close(pl)
        self.plans = []

    # ------------------------------------------------------------ schedule

    def _pos(self, t: int) -> int:
        """Position within the layer of the B block held in phase t."""
        return (self.grid.q + t) % self.lp

    def block_of_phase(self, t: int) -> int:
        """The B block (global index) this rank holds in phase t."""
        return self.grid.layer * self.lp + self._pos(t)

    def _vals(self, vals, l):
        if vals is None:
            return None
        if self.spans[l] is not None:
            return vals.narrow(0, *self.spans[l])
        return vals.index_select(0, self.blocks[l][2])

    # ------------------------------------------------------------ operations

    def fusedmm(self, vals, A_k, B_k):
        """FusedMMA rows of this rank's A block: out_i = sum_j s_ij <A_i, B_j> B_j."""
        g = self.grid
        T = g.gather_fiber(A_k, self.fiber_counts)
        out = torch.empty((self.rows, self.r), dtype=torch.float32, device=A_k.device)
        bufs = _travel_bufs(B_k, self.maxw, self.r, self.dtype, self.lp)
        for t in range(self.lp):
            l = self._pos(t)
            cur = _phase_buf(bufs, t)
            # the next block is in flight while this phase computes
            pend = g.shift(cur, _phase_buf(bufs, t + 1)) if t + 1 < self.lp else []
            # phase 0 writes every output row, later phases add to them
            call = self.ops.fusedmm if t == 0 else self.ops.fusedmm_acc
            call(self.plans[l], self._vals(vals, l), T, cur[:int(self.widths[l])], out)
            g.wait(pend)
        return g.reduce_scatter_fiber(out, self.t_offs)

    def fusedmm_t(self, vals, A_k, B_k):
        """FusedMMB rows of this rank's B block: out_j = sum_i s_ij <A_i, B_j> A_i."""
        g = self.grid
        dev = A_k.device
        T = g.gather_fiber(A_k, self.fiber_counts)
        bufs = _travel_bufs(B_k, self.maxw, self.r, self.dtype, self.lp)
        outs = [torch.empty((self.maxw, self.r), dtype=torch.float32, device=dev)
                for _ in range(1 if self.lp == 1 else 2)]
        cur = 0
        for t in range(self.lp):
            l = self._pos(t)
            b = _phase_buf(bufs, t)
            pend = g.shift(b, _phase_buf(bufs, t + 1)) if t + 1 < self.lp else []
            w = int(self.widths[l])
            call = self.ops.fusedmm_t if t == 0 else self.ops.fusedmm_t_acc
            call(self.plans[l], self._vals(vals, l), T, b[:w], outs[cur][:w])
            if self.lp == 1:
                break
            # the output block travels on with its B block; after p/c shifts
            # it is back at its owner
            g.wait(pend + g.shift(outs[cur], outs[1 - cur]))
            cur = 1 - cur
        return outs[cur][:int(self.widths[g.q])]

    def fusedmm_bwd(self, vals, A_k, B_k, G_k):
        """Adjoint of FusedMMA for L = <G, FusedMMA>: (dA rows of this rank's
        A block, dB rows of its B block, ds of its local nonzeros)."""
        g = self.grid
        dev = A_k.device
        T = g.gather_fiber(A_k, self.fiber_counts)
        TG = g.gather_fiber(G_k, self.fiber_counts)
        dA = torch.empty((self.rows, self.r), dtype=torch.float32, device=dev)
        ds = torch.empty(self.nnz, dtype=torch.float32, device=dev)
        bufs = _travel_bufs(B_k, self.maxw, self.r, self.dtype, self.lp)
        dBs = [torch.empty((self.maxw, self.r), dtype=torch.float32, device=dev)
               for _ in range(1 if self.lp == 1 else 2)]
        cur = 0
        for t in range(self.lp):
            l = self._pos(t)
            b = _phase_buf(bufs, t)
            pend = g.shift(b, _phase_buf(bufs, t + 1)) if t + 1 < self.lp else []
            w = int(self.widths[l])
            sel, span = self.blocks[l][2], self.spans[l]
            ds_l = (ds.narrow(0, *span) if span is not None
                    else torch.empty(sel.numel(), dtype=torch.float32, device=dev))
            call = self.ops.fusedmm_bwd if t == 0 else self.ops.fusedmm_bwd_acc
            call(self.plans[l], self._vals(vals, l), T, b[:w], TG, dA, dBs[cur][:w], ds_l)
            if span is None:
                ds.index_copy_(0, sel, ds_l)
            if self.lp == 1:
                break
            g.wait(pend + g.shift(dBs[cur], dBs[1 - cur]))
            cur = 1 - cur
        return (g.reduce_scatter_fiber(dA, self.t_offs), dBs[cur][:int(self.widths[g.q])], ds)


class ReplicationReuse15D:
    """FusedMMA by replication reuse on the (p/c) x c grid: the B rows of the
    fiber replicated once, then an SDDMM round with the A blocks travelling
    around the layer and an SpMM round with the output blocks travelling.

    Every rank passes its local S = S[R_l, C_q] (row_ptr over the rows R_l
    of its layer's p/c A blocks, int32 col_idx with global columns inside
    the columns C_q of its fiber's c B blocks), n, r, dtype, the A block
    boundaries row_bounds (p + 1) and B block boundaries col_bounds (p + 1,
    default n / p each); then A_k (rows of A block l p/c + q), B_k (rows of
    B block q c + l) and the local values (or None), and gets the FusedMMA
    rows of its A block (float32)."""

    def __init__(self, row_ptr, col_idx, n, r, dtype=torch.float32, row_bounds=None,
                 col_bounds=None, c=1, group=None, ops=None):
        self.grid = Grid15D(c, group)
        g = self.grid
        self.p, self.c, self.lp = g.p, g.c, g.lp
        self.n, self.r, self.dtype = int(n), int(r), dtype
        self.col_bounds = (col_bounds_uniform(self.n, self.p) if col_bounds is None
                           else np.asarray(col_bounds, dtype=np.int64))
        if row_bounds is None:
            raise ValueError("row_bounds (A block boundaries) are needed")
        rb = np.asarray(row_bounds, dtype=np.int64)
        a_lo = g.layer * self.lp
        self.heights = np.diff(rb[a_lo:a_lo + self.lp + 1])
        self.maxh = int(self.heights.max())
        r0 = int(rb[a_lo])
        if row_ptr.numel() - 1 != int(self.heights.sum()):
            raise ValueError("the local S must hold the rows of the layer's A blocks")
        c0 = int(self.col_bounds[g.q * self.c])
        c1 = int(self.col_bounds[(g.q + 1) * self.c])
        self.fiber_counts = np.diff(self.col_bounds[g.q * self.c:(g.q + 1) * self.c + 1])
        if col_idx.numel() and (int(col_idx.min()) < c0 or int(col_idx.max()) >= c1):
            raise ValueError("a column of the local S lies outside its fiber's B blocks")
        self.ops = ops if ops is not None else LibraryOps()
        rp64 = row_ptr.long()
        self.pieces = []   # (plan, first nonzero, nonzeros) per A block of the layer
        for i in range(self.lp):
            lo = int(rb[a_lo + i]) - r0
            hi = int(rb[a_lo + i + 1]) - r0
            p0, p1 = int(rp64[lo]), int(rp64[hi])
            rp = (rp64[lo:hi + 1] - p0).to(torch.int32)
            ci = (col_idx[p0:p1].long() - c0).to(torch.int32)
            self.pieces.append((self.ops.plan(rp, ci, c1 - c0, self.r, dtype), p0, p1 - p0))
        self.nnz = col_idx.numel()

    def close(self):
        for pl, _, _ in self.pieces:
            self.ops.close(pl)
        self.pieces = []

    def _pos(self, t: int) -> int:
        return (self.grid.q + t) % self.lp

    def fusedmm(self, vals, A_k, B_k):
        """FusedMMA rows of this rank's A block."""
        g = self.grid
        dev = A_k.device
        TB = g.gather_fiber(B_k, self.fiber_counts)     # the one replication
        v = torch.empty(self.nnz, dtype=torch.float32, device=dev)
        # round 1: SDDMM values of each piece, the A blocks travelling
        bufs = _travel_bufs(A_k, self.maxh, self.r, self.dtype, self.lp)
        for t in range(self.lp):
            i = self._pos(t)
            plan, p0, cnt = self.pieces[i]
            cur = _phase_buf(bufs, t)
            pend = g.shift(cur, _phase_buf(bufs, t + 1)) if t + 1 < self.lp else []
            vi = None if vals is None else vals.narrow(0, p0, cnt)
            self.ops.sddmm(plan, vi, cur[:int(self.heights[i])], TB, v.narrow(0, p0, cnt))
            g.wait(pend)
        # round 2: SpMM of each piece into the travelling output blocks
        outs = [torch.empty((self.maxh, self.r), dtype=torch.float32, device=dev)
                for _ in range(1 if self.lp == 1 else 2)]
        cur = 0
        for t in range(self.lp):
            i = self._pos(t)
            plan, p0, cnt = self.pieces[i]
            h = int(self.heights[i])
            call = self.ops.spmm if t == 0 else self.ops.spmm_acc
            call(plan, v.narrow(0, p0, cnt), TB, outs[cur][:h])
            if self.lp == 1:
                break
            g.wait(g.shift(outs[cur], outs[1 - cur]))
            cur = 1 - cur
        return outs[cur][:int(self.heights[g.q])]


def slice_bounds(r: int, parts: int) -> np.ndarray:
    """Column slices of the dense width r (parts + 1 boundaries)."""
    return np.array([(k * r) // parts for k in range(parts + 1)], dtype=np.int64)


class SparseShift15D:
    """FusedMMA and FusedMMB by the 1.5D sparse-shifting, dense-replicating
    algorithm (Sec. V) on the (p/c) x c grid: the dense matrices are divided
    by column slices of r, the sparse matrix by block rows, and the block
    rows circulate within each layer.

    S is cut into p block rows balanced by nonzeros; layer l owns the p/c
    consecutive blocks l (p/c) .. (l + 1)(p/c) - 1 (rows R_l), and its p/c
    ranks hold the p/c column slices of r.  Rank (q, l) holds slice q of A's
    rows R_l and of B's columns C_l (B in c blocks of n / c rows); one
    all-gather along the fiber gives it slice q of every row of B (the
    replication, reused by both halves).  Local kernel fusion is impossible
    in this layout (a rank holds only a slice of every row of A and B, so no
    rank can finish a dot product before the aggregation, Sec. IV-B), so
    FusedMM runs as SDDMM then SpMM: round 1 passes each block row's values
    around the layer, every rank adding its slice's partial dot products
    (fmm_sddmm_acc); after p/c phases and p/c shifts each block is back at
    its owner with its SDDMM values complete.  Round 2 passes the completed
    blocks around again, every rank applying each block to its slice
    (fmm_spmm for FusedMMA rows R_l; fmm_spmm_t_acc for FusedMMB, summed over
    the layer's blocks and then reduce-scattered along the fiber, since every
    layer holds part of the rows of S).  The patterns are laid out on every
    rank once (one plan per block row of its layer, at its slice width), so
    only values travel: nnz/p floats per shift.  With c = 1 there is one
    layer holding all rows and every rank all of B's rows.

    Every rank passes the whole pattern (row_ptr, col_idx: int32 on its
    device), the values of all nonzeros (or None), A_k = A[R_l, slice q]
    and B_k = B[C_l, slice q], and gets out[R_l, slice q] (FusedMMA) and
    out_t[C_l, slice q] (FusedMMB)."""

    def __init__(self, row_ptr, col_idx, n, r, dtype=torch.float32, group=None, ops=None,
                 row_bounds=None, c=1):
        self.grid = Grid15D(c, group)
        g = self.grid
        self.p, self.k, self.c, self.lp = g.p, g.k, g.c, g.lp
        self.n, self.r, self.dtype = int(n), int(r), dtype
        self.m = row_ptr.numel() - 1
        self.ops = ops if ops is not None else LibraryOps()
        rp_h = row_ptr.cpu().numpy()
        self.row_bounds = (row_bounds_by_nnz(rp_h, self.p) if row_bounds is None
                           else np.asarray(row_bounds, dtype=np.int64))
        self.slices = slice_bounds(self.r, self.lp)
        self.width = int(self.slices[g.q + 1] - self.slices[g.q])
        self.nnz_bounds = rp_h.astype(np.int64)[self.row_bounds]
        # this layer's block rows and rows, and the fiber's blocks of B
        self.b0 = g.layer * self.lp
        self.r_lo = int(self.row_bounds[self.b0])
        self.r_hi = int(self.row_bounds[self.b0 + self.lp])
        self.col_bounds = col_bounds_uniform(self.n, self.c)
        self.plans = []
        for i in range(self.lp):
            b = self.b0 + i
            r0, r1 = int(self.row_bounds[b]), int(self.row_bounds[b + 1])
            p0, p1 = int(self.nnz_bounds[b]), int(self.nnz_bounds[b + 1])
            rp = (row_ptr[r0:r1 + 1].long() - p0).to(torch.int32)
            self.plans.append(self.ops.plan(rp, col_idx[p0:p1], self.n, self.width, dtype))
        self.maxnz = int(np.diff(self.nnz_bounds).max()) if self.p else 0

    def close(self):
        for pl in self.plans:
            self.ops.close(pl)
        self.plans = []

    def block_of_phase(self, t: int) -> int:
        """The block row (global index) whose values this rank holds in phase t."""
        return self.b0 + (self.grid.q + t) % self.lp

    def _rows(self, b):
        return int(self.row_bounds[b]), int(self.row_bounds[b + 1])

    def _nz(self, b):
        return int(self.nnz_bounds[b]), int(self.nnz_bounds[b + 1])

    def _sddmm_round(self, vals, A_k, TB):
        """Round 1: every block row's SDDMM values, summed over the layer's
        slices; returns (the value buffers, the current one: this rank's
        own block, complete)."""
        g = self.grid
        dev = A_k.device
        bufs = [torch.zeros(self.maxnz, dtype=torch.float32, device=dev),
                torch.empty(self.maxnz, dtype=torch.float32, device=dev)]
        cur = 0
        for t in range(self.lp):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            v = None if vals is None else vals[p0:p1]
            self.ops.sddmm_acc(self.plans[b - self.b0], v, A_k[r0 - self.r_lo:r1 - self.r_lo], TB,
                               bufs[cur][:p1 - p0])
            g.wait(g.shift(bufs[cur], bufs[1 - cur]))
            cur = 1 - cur
        return bufs, cur

    def _replicated_b(self, B_k):
        return self.grid.gather_fiber(B_k, np.diff(self.col_bounds))

    def fusedmm(self, vals, A_k, B_k):
        """out[R_l, slice q] of FusedMMA ((r_hi - r_lo) x r_q)."""
        g = self.grid
        TB = self._replicated_b(B_k)
        bufs, cur = self._sddmm_round(vals, A_k, TB)
        out = torch.empty((self.r_hi - self.r_lo, self.width), dtype=torch.float32,
                          device=A_k.device)
        for t in range(self.lp):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            pend = g.shift(bufs[cur], bufs[1 - cur]) if t + 1 < self.lp else []
            self.ops.spmm(self.plans[b - self.b0], bufs[cur][:p1 - p0], TB,
                          out[r0 - self.r_lo:r1 - self.r_lo])
            g.wait(pend)
            cur = 1 - cur
        return out

    def fusedmm_t(self, vals, A_k, B_k):
        """out_t[C_l, slice q] of FusedMMB."""
        g = self.grid
        TB = self._replicated_b(B_k)
        bufs, cur = self._sddmm_round(vals, A_k, TB)
        part = torch.zeros((self.n, self.width), dtype=torch.float32, device=A_k.device)
        for t in range(self.lp):
            b = self.block_of_phase(t)
            (r0, r1), (p0, p1) = self._rows(b), self._nz(b)
            pend = g.shift(bufs[cur], bufs[1 - cur]) if t + 1 < self.lp else []
            self.ops.spmm_t_acc(self.plans[b - self.b0], bufs[cur][:p1 - p0],
                                A_k[r0 - self.r_lo:r1 - self.r_lo], part)
            g.wait(pend)
            cur = 1 - cur
        # every layer summed its rows: the sum over the fiber, scattered
        return g.reduce_scatter_fiber(part, self.col_bounds)
