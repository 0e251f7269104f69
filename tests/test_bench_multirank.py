"""The multi-rank parts of bench.py on CPU: two gloo ranks, max-over-ranks
timing and the whole-job throughput formula (no GPU involved)."""
import json
import os
import socket
import sys

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


def _bench(env_extra, *args):
    import subprocess
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "1", "--scale", "0.25", "--steps", "1", "--warmup", "3",
                           *args], capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_prints_on_rank_zero_only():
    """The reference arm (the FP64 oracle on host cores) runs on rank 0; under
    torchrun the other ranks exit 0 without work and print nothing."""
    other = _bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert other.returncode == 0, other.stderr
    assert other.stdout.strip() == ""
    first = _bench({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert first.returncode == 0, first.stderr
    lines = [line for line in first.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench_unit()
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k


def bench_unit():
    sys.path.insert(0, ROOT)
    import bench
    return bench.UNIT
