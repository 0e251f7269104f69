#!/usr/bin/env python3
"""FusedMM benchmark: one JSON line with throughput, roofline and baselines.

A step is one pass of the hot path over the workload: FusedMMA (fmm_fusedmm)
and FusedMMB (fmm_fusedmm_t) on an Erdos-Renyi pattern with m = n = 2^20,
exactly 32 nonzeros per row (~33.5M), r = 128, float32, s ~ U(0,1),
A, B ~ N(0, 1/128).  The metric counts nnz * r per FusedMM call, so one step
is 2 * nnz * r units.  Beside it the unfused path (SDDMM writes v, SpMM reads
it) is timed on the same inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..4]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)

Under torchrun each rank runs its own replica (weak scaling: the path has no
exchange step); value = units of all ranks / max-over-ranks time.
Timing: CUDA events on the launching stream, barrier + synchronize on both
sides; inputs (A, B: 512 MiB each) are larger than L2, so L2 is not flushed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("FusedMM nnz·r/s and HBM GB/s vs peak; fused vs unfused SDDMM→SpMM, "
          "same GPU")
UNIT = "nnz*r/s"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "roofline_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2203_07673_gb300", "csrc", f)
                  for f in ("fmm_rows.cuh", "fmm_rows_f32.cu", "fmm_rows_bf16.cu",
                            "fmm_internal.cuh")]


def kernel_source_sha() -> str:
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def gather_model_bytes(m, nnz, r, e, vals=True):
    """Algorithmic bytes of one FusedMM call: the CSR (row_ptr, col_idx,
    values), each local row read once (rows x r x e), one dense row gathered
    per nonzero (nnz x r x e) and the float32 output written once."""
    return 4 * (m + 1) + 4 * nnz + (4 * nnz if vals else 0) + m * r * e + nnz * r * e + 4 * m * r


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(k: int, scale: float):
    from paper_2203_07673_gb300 import workloads as wl
    return wl.workload(k, scale_rows=scale)


# --------------------------------------------------------------- oracle leg

def oracle_sample(w, seconds: float, rows_hint: int | None = None):
    """Times the FP64 oracle (FusedMMA + FusedMMB) on the first rows of the
    workload, columns remapped to the ones those rows touch.  Returns
    (units per second, description, threads)."""
    import oracle
    S, r = w["S"], w["r"]
    A = w["A"].astype(np.float64) if w["dtype"] == "f32" else _bf16_round(w["A"])
    B = w["B"].astype(np.float64) if w["dtype"] == "f32" else _bf16_round(w["B"])
    vals = None if w["vals"] is None else w["vals"].astype(np.float64)

    def sub(rows):
        sub_s = S.rows_slice(0, rows)
        cols, ci = np.unique(sub_s.col_idx, return_inverse=True)
        v = None if vals is None else vals[:sub_s.nnz]
        return sub_s.row_ptr, ci.astype(np.int64), v, A[:rows], B[cols], len(cols), sub_s.nnz

    def run(rows):
        rp, ci, v, a, b, n, nnz = sub(rows)
        t0 = time.perf_counter()
        oracle.fusedmm(rp, ci, v, a, b, n)
        oracle.fusedmm_t(rp, ci, v, a, b, n)
        return time.perf_counter() - t0, nnz, n

    rows = rows_hint or min(S.m, 1024)
    t, nnz, ncols = run(rows)
    if rows_hint is None:
        rows = int(min(S.m, max(rows, rows * seconds / max(t, 1e-6))))
        t, nnz, ncols = run(rows)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"first {rows} of {S.m} rows ({nnz} nnz, {nnz / max(S.nnz, 1):.2%} of the "
            f"workload), columns remapped to the {ncols} they touch; "
            f"FusedMMA + FusedMMB in FP64 (oracle/fmm_oracle.c); FusedMMA rows on "
            f"{threads} OpenMP threads, the FusedMMB scatter on 1")
    return 2.0 * nnz * r / t, desc, threads, rows


def _bf16_round(x):
    import torch
    return torch.from_numpy(x).to(torch.bfloat16).double().numpy()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = make_workload(args.workload, args.scale)
    # calibrate one step to about 1 s of CPU work, then time W + K steps
    _, _, _, rows = oracle_sample(w, 1.0)
    for _ in range(args.warmup):
        oracle_sample(w, 1.0, rows_hint=rows)
    vals, desc = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc, threads, _ = oracle_sample(w, 1.0, rows_hint=rows)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(w, args):
    S = w["S"]
    return {"workload": w["name"], "m": S.m, "n": S.n, "nnz": S.nnz, "r": w["r"],
            "input_dtype": w["dtype"], "step": "FusedMMA + FusedMMB",
            "l2": "not flushed: A and B are larger than L2" if S.m * w["r"] * 4 > 2**28
            else "L2-resident inputs", "parallelism": f"replicas x{args.gpus}",
            "scale_rows": args.scale}


# ------------------------------------------------------------------ GPU leg

def run_fmm(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2203_07673_gb300 import fmm

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, args.scale)
    S, r = w["S"], w["r"]
    tdt = torch.float32 if w["dtype"] == "f32" else torch.bfloat16
    e = 4 if w["dtype"] == "f32" else 2
    rp = torch.from_numpy(S.row_ptr).to(dev)
    ci = torch.from_numpy(S.col_idx).to(dev)
    vals = None if w["vals"] is None else torch.from_numpy(w["vals"]).to(dev)
    A = torch.from_numpy(w["A"]).to(dev).to(tdt).contiguous()
    B = torch.from_numpy(w["B"]).to(dev).to(tdt).contiguous()
    plan = fmm.Plan(rp, ci, S.n, r, tdt)
    info = plan.info()
    out = torch.empty(S.m, r, device=dev)
    out_t = torch.empty(S.n, r, device=dev)
    v = torch.empty(S.nnz, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        fmm.fusedmm(plan, vals, A, B, out=out)
        fmm.fusedmm_t(plan, vals, A, B, out=out_t)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        fmm.fusedmm(plan, vals, A, B, out=out)
        ev[k][1].record(stream)
        fmm.fusedmm_t(plan, vals, A, B, out=out_t)
        ev[k][2].record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    fwd_ms = float(np.mean([ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]))
    fwd_t_ms = float(np.mean([ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]))
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    # unfused path (SDDMM writes v, SpMM reads it back), same inputs
    def unfused():
        fmm.sddmm(plan, vals, A, B, out=v)
        fmm.spmm(plan, v, B, out=out)
        fmm.sddmm(plan, vals, A, B, out=v)
        fmm.spmm_t(plan, v, A, out=out_t)

    for _ in range(max(1, args.warmup)):
        unfused()
    barrier()
    u0 = torch.cuda.Event(enable_timing=True); u1 = torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    for _ in range(K):
        unfused()
    u1.record(stream)
    barrier()
    unfused_ms = u0.elapsed_time(u1) / K

    # end to end through the public API from pinned host buffers
    A_h = torch.from_numpy(w["A"]).to(tdt).pin_memory()
    B_h = torch.from_numpy(w["B"]).to(tdt).pin_memory()
    vals_h = None if w["vals"] is None else torch.from_numpy(w["vals"]).pin_memory()
    out_h = torch.empty(S.m, r).pin_memory()
    out_t_h = torch.empty(S.n, r).pin_memory()

    def e2e_step():
        A.copy_(A_h, non_blocking=True)
        B.copy_(B_h, non_blocking=True)
        if vals is not None:
            vals.copy_(vals_h, non_blocking=True)
        fmm.fusedmm(plan, vals, A, B, out=out)
        fmm.fusedmm_t(plan, vals, A, B, out=out_t)
        out_h.copy_(out, non_blocking=True)
        out_t_h.copy_(out_t, non_blocking=True)

    for _ in range(max(1, min(args.warmup, 3))):
        e2e_step()
    barrier()
    k_e2e = max(1, min(K, 50))
    x0 = torch.cuda.Event(enable_timing=True); x1 = torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(k_e2e):
        e2e_step()
    x1.record(stream)
    barrier()
    e2e_ms = x0.elapsed_time(x1) / k_e2e
    if world > 1:
        t = torch.tensor([unfused_ms, e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        unfused_ms, e2e_ms = (float(x) for x in t.tolist())

    units_step = 2.0 * S.nnz * r
    value = units_step * K * world / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / K
    peak, peak_kind = load_peaks()
    alg = gather_model_bytes(S.m, S.nnz, r, e, vals is not None)
    achieved = alg / (fwd_ms / 1e3) / 1e9
    traffic, traffic_note = None, "no ncu capture for the current kernel source"
    try:
        with open(PROFILE_TRAFFIC) as fh:
            prof = json.load(fh)
        if (prof.get("source_sha1") == kernel_source_sha()
                and prof.get("workload") == w["name"]):
            traffic = float(prof["dram_bytes_per_launch"])
            traffic_note = prof.get("note", "")
    except Exception:
        pass
    launches_per_call = 1 + (1 if info["split_rows"] else 0)
    launches_per_call_t = 1 + (1 if info["split_cols"] else 0) + (1 if vals is not None else 0)
    h2d = A_h.numel() * A_h.element_size() + B_h.numel() * B_h.element_size() + (
        0 if vals_h is None else vals_h.numel() * 4)
    d2h = (out_h.numel() + out_t_h.numel()) * 4

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, args),
        "roofline": {
            "bound": "hbm", "kernel": "row_pass_kernel<M_FUSED> (fmm_fusedmm)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
            "algorithmic_bytes_per_launch": alg,
            "bytes_model": "gather model: CSR + local rows once + one dense row per nonzero "
                           "+ float32 output once",
            "kernel_ms": fwd_ms,
            "dram_frac": None if traffic is None else traffic / (fwd_ms / 1e3) / 1e9 / peak,
            "traffic_note": traffic_note,
        },
        "fused": {"fusedmm_ms": fwd_ms, "fusedmm_t_ms": fwd_t_ms,
                  "unfused_ms_per_step": unfused_ms,
                  "fused_speedup_vs_unfused": unfused_ms / ms_per_step},
        "e2e": {"value": units_step * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": K * (launches_per_call + launches_per_call_t),
        "clocks": clk,
        "plan": {k: info[k] for k in ("max_row_nnz", "max_col_nnz", "split_rows",
                                      "split_cols", "variant", "variant_t",
                                      "workspace_bytes")},
    }
    if rank == 0 and not args.no_cpu_baseline:
        cv, desc, threads, _ = oracle_sample(w, args.cpu_seconds)
        line["cpu_baseline"] = {"value": cv, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fmm", "reference"], default="fmm")
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--scale", type=float, default=1.0, help="row-count scale (1 = full)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    rc = run_fmm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
