"""The multi-rank parts of bench.py on CPU: two gloo ranks, max-over-ranks
timing and the whole-job throughput formula (no GPU involved)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.reduce_max([10.0 * (rank + 1), 5.0 - rank], "cpu", world)
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_reduce_max_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == [20.0, 5.0] and out[1] == [20.0, 5.0]


def test_whole_job_value_formula():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 10 steps x 100 units, slowest rank 4 ms -> 2000 units / 0.004 s
    assert bench.whole_job_value(100.0, 10, 2, 4.0) == pytest.approx(5e5)
    assert bench.reduce_max([1.0, 2.0], "cpu", 1) == [1.0, 2.0]
