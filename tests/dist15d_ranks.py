"""Rank bodies of the 1.5D FusedMM tests (Sec. V, Algorithm 1, c = 1), run in
spawned processes by tests/test_dist15d.py and tests/test_gpu_dist15d.py.

Every rank draws the same seeded whole problem, keeps its own row block of S
and A and its own block of B, runs FusedMMA, FusedMMB and the FusedMMA
adjoint through paper_2203_07673_gb300.dist15d, and returns its blocks of
the results; the parent assembles them and compares them with the oracle on
the whole matrix.  `OracleOps` is the local-kernel stand-in of the CPU test:
it evaluates each local call with the FP64 oracle (test infrastructure; the
product never imports the oracle)."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))


def problem(seed, m=300, n=250, r=32):
    from paper_2203_07673_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    S = wl.random_csr(m, n, rng, mean_deg=6, empty_frac=0.1, hubs=((7, 180), (m - 1, 90)))
    vals = rng.uniform(0.5, 1.5, S.nnz).astype(np.float32)
    A = (rng.standard_normal((m, r)) / np.sqrt(r)).astype(np.float32)
    B = (rng.standard_normal((n, r)) / np.sqrt(r)).astype(np.float32)
    G = rng.standard_normal((m, r)).astype(np.float32)
    return S, vals, A, B, G


class OracleOps:
    """Local calls of the 1.5D driver evaluated by the FP64 oracle (CPU)."""

    def __init__(self):
        import oracle
        self.o = oracle

    def plan(self, row_ptr, col_idx, n, r, dtype):
        return dict(rp=row_ptr.cpu().numpy(), ci=col_idx.cpu().numpy(), n=int(n))

    @staticmethod
    def _np(x):
        return None if x is None else x.detach().cpu().double().numpy()

    def fusedmm(self, plan, vals, A, B, out):
        out.zero_()
        self.fusedmm_acc(plan, vals, A, B, out)

    def fusedmm_t(self, plan, vals, A, B, out):
        out.zero_()
        self.fusedmm_t_acc(plan, vals, A, B, out)

    def fusedmm_bwd(self, plan, vals, A, B, G, dA, dB, ds):
        dA.zero_(); dB.zero_()
        self.fusedmm_bwd_acc(plan, vals, A, B, G, dA, dB, ds)

    def fusedmm_acc(self, plan, vals, A, B, out):
        res = self.o.fusedmm(plan["rp"], plan["ci"], self._np(vals), self._np(A), self._np(B),
                             plan["n"])
        out += torch.from_numpy(res).to(out.dtype)

    def fusedmm_t_acc(self, plan, vals, A, B, out):
        res = self.o.fusedmm_t(plan["rp"], plan["ci"], self._np(vals), self._np(A), self._np(B),
                               plan["n"])
        out += torch.from_numpy(res).to(out.dtype)

    def fusedmm_bwd_acc(self, plan, vals, A, B, G, dA, dB, ds):
        ga, gb, gs = self.o.fusedmm_grad(plan["rp"], plan["ci"], self._np(vals), self._np(A),
                                         self._np(B), self._np(G), plan["n"])
        dA += torch.from_numpy(ga).to(dA.dtype)
        dB += torch.from_numpy(gb).to(dB.dtype)
        ds.copy_(torch.from_numpy(gs).to(ds.dtype))

    def sddmm(self, plan, vals, A, B, v):
        v.zero_()
        self.sddmm_acc(plan, vals, A, B, v)

    def spmm_acc(self, plan, v, B, out):
        res = self.o.spmm(plan["rp"], plan["ci"], self._np(v), self._np(B), plan["n"])
        out += torch.from_numpy(res).to(out.dtype)

    def sddmm_acc(self, plan, vals, A, B, v):
        res = self.o.sddmm(plan["rp"], plan["ci"], self._np(vals), self._np(A), self._np(B),
                           plan["n"])
        v += torch.from_numpy(res).to(v.dtype)

    def spmm(self, plan, v, B, out):
        res = self.o.spmm(plan["rp"], plan["ci"], self._np(v), self._np(B), plan["n"])
        out.copy_(torch.from_numpy(res).to(out.dtype))

    def spmm_t_acc(self, plan, v, A, out):
        res = self.o.spmm_t(plan["rp"], plan["ci"], self._np(v), self._np(A), plan["n"])
        out += torch.from_numpy(res).to(out.dtype)

    def close(self, plan):
        pass


def rank_main(rank, world, port, out, seed, r, use_gpu, vals_none, c=1, bf16=False):
    """FusedMM15D on the (world/c) x c grid: the rank's local S = S[T_q, C_l],
    A block q c + l, B block l (world/c) + q; with bf16, A and B in bfloat16
    (the blocks moved along fibers and rings as raw bytes)."""
    import torch.distributed as dist
    from paper_2203_07673_gb300 import dist15d
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S, vals, A, B, G = problem(seed, r=r)
        rb = dist15d.row_bounds_by_nnz(S.row_ptr, world)
        cb = dist15d.col_bounds_uniform(S.n, world)
        lp = world // c
        layer, q = divmod(rank, lp)
        a, b = q * c + layer, layer * lp + q
        rp_l, ci_l, slots = dist15d.local_block(
            torch.from_numpy(S.row_ptr), torch.from_numpy(S.col_idx), int(rb[q * c]),
            int(rb[(q + 1) * c]), int(cb[layer * lp]), int(cb[(layer + 1) * lp]))
        r0, r1, c0, c1 = int(rb[a]), int(rb[a + 1]), int(cb[b]), int(cb[b + 1])
        dev = torch.device("cuda", 0) if use_gpu else torch.device("cpu")
        rp, ci = rp_l.to(dev), ci_l.to(dev)
        vk = None if vals_none else torch.from_numpy(vals[slots.numpy()]).to(dev)
        dt = torch.bfloat16 if bf16 else torch.float32
        Ak = torch.from_numpy(A[r0:r1].copy()).to(dev).to(dt)
        Bk = torch.from_numpy(B[c0:c1].copy()).to(dev).to(dt)
        Gk = torch.from_numpy(G[r0:r1].copy()).to(dev)
        ops = None if use_gpu else OracleOps()
        d = dist15d.FusedMM15D(rp, ci, S.n, r, dt, ops=ops, c=c, row_bounds=rb)
        assert [d.block_of_phase(t) for t in range(lp)] == [layer * lp + (q + t) % lp
                                                            for t in range(lp)]
        B_in = Bk.clone()
        res = dict(out=d.fusedmm(vk, Ak, Bk), out_t=d.fusedmm_t(vk, Ak, Bk))
        res["dA"], res["dB"], res["ds"] = d.fusedmm_bwd(vk, Ak, Bk, Gk)
        if use_gpu:
            torch.cuda.synchronize()
        # the rank's B block is sent in phase 0 but never received into
        assert torch.equal(Bk, B_in)
        out[rank] = {k: v.cpu().numpy() for k, v in res.items()}
        out[f"bounds{rank}"] = (r0, r1, c0, c1, slots.numpy())
        d.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def reuse_rank_main(rank, world, port, out, seed, r, use_gpu, vals_none, c=1):
    """ReplicationReuse15D on the (world/c) x c grid: the rank's local S =
    S[R_l, C_q], A block l (world/c) + q, B block q c + l."""
    import torch.distributed as dist
    from paper_2203_07673_gb300 import dist15d
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S, vals, A, B, G = problem(seed, r=r)
        rb = dist15d.row_bounds_by_nnz(S.row_ptr, world)
        cb = dist15d.col_bounds_uniform(S.n, world)
        lp = world // c
        layer, q = divmod(rank, lp)
        a, b = layer * lp + q, q * c + layer
        rp_l, ci_l, slots = dist15d.local_block(
            torch.from_numpy(S.row_ptr), torch.from_numpy(S.col_idx), int(rb[layer * lp]),
            int(rb[(layer + 1) * lp]), int(cb[q * c]), int(cb[(q + 1) * c]))
        r0, r1, c0, c1 = int(rb[a]), int(rb[a + 1]), int(cb[b]), int(cb[b + 1])
        dev = torch.device("cuda", 0) if use_gpu else torch.device("cpu")
        vk = None if vals_none else torch.from_numpy(vals[slots.numpy()]).to(dev)
        Ak = torch.from_numpy(A[r0:r1].copy()).to(dev)
        Bk = torch.from_numpy(B[c0:c1].copy()).to(dev)
        ops = None if use_gpu else OracleOps()
        d = dist15d.ReplicationReuse15D(rp_l.to(dev), ci_l.to(dev), S.n, r, torch.float32,
                                        row_bounds=rb, c=c, ops=ops)
        A_in = Ak.clone()
        res = dict(out=d.fusedmm(vk, Ak, Bk))
        if use_gpu:
            torch.cuda.synchronize()
        assert torch.equal(Ak, A_in)
        out[rank] = {k: v.cpu().numpy() for k, v in res.items()}
        out[f"bounds{rank}"] = (r0, r1)
        d.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def sparse_rank_main(rank, world, port, out, seed, r, use_gpu, vals_none, c=1):
    """The sparse-shifting algorithm on the (world/c) x c grid: every rank
    holds the whole pattern and values, A[R_l, slice q] and B[C_l, slice q];
    returns out[R_l, slice q] and out_t[C_l, slice q]."""
    import torch.distributed as dist
    from paper_2203_07673_gb300 import dist15d
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S, vals, A, B, G = problem(seed, r=r)
        lp = world // c
        layer, q = divmod(rank, lp)
        sl = dist15d.slice_bounds(r, lp)
        j0, j1 = int(sl[q]), int(sl[q + 1])
        rb = dist15d.row_bounds_by_nnz(S.row_ptr, world)
        r0, r1 = int(rb[layer * lp]), int(rb[(layer + 1) * lp])
        cb = dist15d.col_bounds_uniform(S.n, c)
        c0, c1 = int(cb[layer]), int(cb[layer + 1])
        dev = torch.device("cuda", 0) if use_gpu else torch.device("cpu")
        rp = torch.from_numpy(S.row_ptr.copy()).to(dev)
        ci = torch.from_numpy(S.col_idx.copy()).to(dev)
        vt = None if vals_none else torch.from_numpy(vals).to(dev)
        Ak = torch.from_numpy(np.ascontiguousarray(A[r0:r1, j0:j1])).to(dev)
        Bk = torch.from_numpy(np.ascontiguousarray(B[c0:c1, j0:j1])).to(dev)
        ops = None if use_gpu else OracleOps()
        d = dist15d.SparseShift15D(rp, ci, S.n, r, torch.float32, ops=ops, c=c)
        res = dict(out=d.fusedmm(vt, Ak, Bk), out_t=d.fusedmm_t(vt, Ak, Bk))
        if use_gpu:
            torch.cuda.synchronize()
        out[rank] = {k: v.cpu().numpy() for k, v in res.items()}
        out[f"slice{rank}"] = (j0, j1, r0, r1, c0, c1)
        d.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()
