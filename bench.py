#!/usr/bin/env python3
"""FusedMM benchmark: one JSON line with throughput, roofline and baselines.

A step is one pass of the hot path over the workload: FusedMMA (fmm_fusedmm)
and FusedMMB (fmm_fusedmm_t) on an Erdos-Renyi pattern with m = n = 2^20,
exactly 32 nonzeros per row (~33.5M), r = 128, float32, s ~ U(0,1),
A, B ~ N(0, 1/128).  The metric counts nnz * r per FusedMM call, so one step
is 2 * nnz * r units.  Beside it the unfused path (SDDMM writes v, SpMM reads
it) is timed on the same inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..5] [--bf16]
  python bench.py --als | --gat [--gat-bf16]   (ALS sweeps; graph-attention forward)
  python bench.py --impl reference ...          (the FP64 CPU oracle on host cores)

Workloads: 1 ER 4096^2 (r = 32), 2 ER 2^20 (r = 128, the default), 3 R-MAT
2^22 forward + backward (BF16), 4 Zipf rows 2^21 x 2^19 (r = 64; --bf16 for
BF16 A and B), 5 512 uneven matrices in one persistent launch per phase.

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
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2203_07673_gb300", "csrc", f)
                  for f in ("fmm_rows.cuh", "fmm_rows_f32.cu", "fmm_rows_bf16.cu",
                            "fmm_staged.cuh", "fmm_staged_f32.cu", "fmm_staged_bf16.cu",
                            "fmm_pipe.cuh", "fmm_pipe_f32.cu", "fmm_pipe_bf16.cu",
                            "fmm_stream.cuh", "fmm_stream_f32.cu", "fmm_stream_bf16.cu",
                            "fmm_internal.cuh", "fmm_plan.cu")]


GAT_SOURCES = [os.path.join(ROOT, "paper_2203_07673_gb300", "csrc", f)
               for f in ("fmm_gat.cu", "fmm_rows.cuh", "fmm_internal.cuh", "fmm_plan.cu")]


def kernel_source_sha(call: str = "") -> str:
    h = hashlib.sha1()
    for f in (GAT_SOURCES if call == "fmm_gat_forward" else KERNEL_SOURCES):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def read_traffic(workload, call, dtype):
    """DRAM bytes per call from profiles/roofline_traffic.txt, if captured on
    the current kernel sources; else (None, reason)."""
    try:
        sha = kernel_source_sha(call)
        with open(PROFILE_TRAFFIC) as fh:
            for line in fh:
                if line.startswith("#") or "|" not in line:
                    continue
                f = [x.strip() for x in line.split("|")]
                if f[0] == workload and f[1] == call and f[2] == dtype:
                    if f[4] != sha:
                        return None, "ncu capture predates the current kernel source"
                    return float(f[3]), f[5]
    except OSError:
        pass
    return None, "no ncu capture for this workload and call"


def gather_model_bytes(m, nnz, r, e, vals=True):
    """Algorithmic bytes of one FusedMM row pass: the CSR (row_ptr, col_idx,
    values), each local row read once (rows x r x e), one dense row gathered
    per nonzero (nnz x r x e) and the float32 output written once."""
    return 4 * (m + 1) + 4 * nnz + (4 * nnz if vals else 0) + m * r * e + nnz * r * e + 4 * m * r


def compulsory_model_bytes(m, n, nnz, r, e, vals=True):
    """The same pass if every dense row were read from DRAM once: the
    gathers are replaced by the n x r x e bytes of the gathered matrix."""
    return 4 * (m + 1) + 4 * nnz + (4 * nnz if vals else 0) + m * r * e + n * r * e + 4 * m * r


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal


def permute_bytes(nnz):
    """Values of S into S^T order: perm read, one value fetched, one written."""
    return 12 * nnz


def gather_model_bytes_mn(m, n, nnz, r, e, vals=True):
    return gather_model_bytes(m, nnz, r, e, vals)


def step_calls(k, S, r, e, vals_given, model=gather_model_bytes_mn):
    """(name, model bytes) of the calls of one step of workload k, by the
    gather model (default) or compulsory_model_bytes."""
    return _calls(k, S.m, S.n, S.nnz, r, e, vals_given, model)


def _calls(k, m, n, nnz, r, e, vals_given, model):
    fwd = model(m, n, nnz, r, e, vals_given)
    fwd_t = model(n, m, nnz, r, e, vals_given) + (permute_bytes(nnz) if vals_given else 0)
    if k == 3:
        # backward: pass over S (A_i, G_i local, B_j gathered, dA and ds written),
        # pass over S^T (B_j local, A_i and G_i gathered, dB written)
        p1 = model(m, n, nnz, r, e, vals_given) + 4 * m * r + 4 * nnz
        g_rows = nnz if model is gather_model_bytes_mn else m   # G_i with each gathered A_i
        p2 = model(n, m, nnz, r, e, vals_given) + 4 * g_rows * r + (
            permute_bytes(nnz) if vals_given else 0)
        return [("fmm_fusedmm", fwd), ("fmm_fusedmm_bwd", p1 + p2)]
    return [("fmm_fusedmm", fwd), ("fmm_fusedmm_t", fwd_t)]


def reduce_max(values, device, world):
    """Element-wise maximum of a list of floats over all ranks."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_value(units_per_step_per_rank, steps, world, max_elapsed_ms):
    """Units all ranks processed divided by the slowest rank's time (per s)."""
    return units_per_step_per_rank * steps * world / (max_elapsed_ms / 1e3)


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

    log_path = None   # --clock-log: keep the raw samples here (else a temporary file)

    def __init__(self, device_index: int):
        import tempfile
        self.proc = None
        self.dev = device_index
        self.path = (ClockSampler.log_path + f".rank{device_index}.csv" if ClockSampler.log_path
                     else os.path.join(tempfile.gettempdir(),
                                       f"fmm_clocks_{os.getpid()}_rank{device_index}.csv"))

    def start(self):
        try:
            if os.path.dirname(self.path):
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


def make_workload(k: int, scale: float, bf16: bool = False):
    """Workload k; bf16 runs the FP32 workloads (2, 4) with A and B rounded
    to bfloat16 (the BF16 case of the Zipf-row configuration)."""
    from paper_2203_07673_gb300 import workloads as wl
    w = wl.workload(k, scale_rows=scale)
    w["k"] = k
    if bf16 and w["dtype"] == "f32":
        w["dtype"] = "bf16"
        w["name"] = w["name"] + " [BF16 A,B]"
    return w


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

    fwd_bwd = w.get("k") == 3

    def run(rows):
        rp, ci, v, a, b, n, nnz = sub(rows)
        t0 = time.perf_counter()
        oracle.fusedmm(rp, ci, v, a, b, n)
        if fwd_bwd:
            oracle.fusedmm_grad(rp, ci, v if v is not None else np.ones(nnz), a, b, a, n)
        else:
            oracle.fusedmm_t(rp, ci, v, a, b, n)
        return time.perf_counter() - t0, nnz, n

    rows = rows_hint or min(S.m, 1024)
    t, nnz, ncols = run(rows)
    if rows_hint is None:
        rows = int(min(S.m, max(rows, rows * seconds / max(t, 1e-6))))
        t, nnz, ncols = run(rows)
    threads = oracle.threads()
    what = ("FusedMMA forward (rows on {t} OpenMP threads) + its gradient (sequential)"
            if fwd_bwd else "FusedMMA (rows on {t} OpenMP threads) + FusedMMB (sequential scatter)")
    desc = (f"first {rows} of {S.m} rows ({nnz} nnz, {nnz / max(S.nnz, 1):.2%} of the "
            f"workload), columns remapped to the {ncols} they touch; "
            + what.format(t=threads) + " in FP64 (oracle/fmm_oracle.c)")
    return (1.0 if fwd_bwd else 2.0) * nnz * r / t, desc, threads, rows


def single_thread_oracle(w, seconds):
    """The oracle sample again on one thread (a smaller sample)."""
    import oracle
    before = oracle.threads()
    try:
        oracle.threads(1)
        v, _, _, rows = oracle_sample(w, seconds)
    finally:
        oracle.threads(before)
    return {"single_thread_value": v, "single_thread_rows": rows}


def _bf16_round(x):
    import torch
    return torch.from_numpy(x).to(torch.bfloat16).double().numpy()


def batched_oracle_step(mats, seconds):
    """FP64 oracle FusedMMA + gradient over the batched matrices in order
    until `seconds` of CPU time; returns (units per second, matrices used)."""
    import oracle
    units, spent, used = 0.0, 0.0, 0
    for m in mats:
        if spent >= seconds:
            break
        S, r = m["S"], m["r"]
        a = _bf16_round(m["A"]); b = _bf16_round(m["B"])
        v = m["vals"].astype(np.float64)
        t0 = time.perf_counter()
        oracle.fusedmm(S.row_ptr, S.col_idx, v, a, b, S.n)
        oracle.fusedmm_grad(S.row_ptr, S.col_idx, v, a, b, a, S.n)
        spent += time.perf_counter() - t0
        units += S.nnz * r
        used += 1
    return units / spent, used


def run_reference_batched(args):
    from paper_2203_07673_gb300 import workloads as wl
    specs = wl.batched_specs(args.batch_count, scale_rows=args.scale)
    mats = []
    for t, sp in enumerate(specs[:64]):
        mats.append(wl.batched_matrix(sp, t))
    for _ in range(args.warmup):
        batched_oracle_step(mats, 0.5)
    vals, used = [], 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, used = batched_oracle_step(mats, 1.0)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.median(vals))
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"the first {used} of {len(specs)} batched matrices (numpy-drawn, same recipe), "
            f"FusedMMA (rows on {threads} OpenMP threads) + its gradient (sequential) in FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.WORKLOADS[5]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    if args.workload == 5:
        return run_reference_batched(args)
    w = make_workload(args.workload, args.scale, args.bf16)
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


def serial_e2e(compute, host_in, slot_in, host_out, slot_out):
    """One end-to-end step on the current stream: uploads, compute, read-backs."""
    for h, d in zip(host_in, slot_in[0]):
        if h is not None:
            d.copy_(h, non_blocking=True)
    compute(0)
    for h, d in zip(host_out, slot_out[0]):
        h.copy_(d, non_blocking=True)


def pipelined_e2e(compute, host_in, slot_in, host_out, slot_out, reps, warmup, barrier):
    """Milliseconds per end-to-end step with double buffering: step i uploads
    its inputs into slot i % 2 on an upload stream, computes on the current
    stream and reads its outputs back on a read-back stream; a slot is
    reused only after its previous step's compute and read-back finished.
    Every step moves all its inputs and outputs inside the timed region."""
    import torch
    main = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    in_ready, done, out_free = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    used = [False, False]

    def step(i):
        slot = i % 2
        if used[slot]:
            s_in.wait_event(done[slot])
        with torch.cuda.stream(s_in):
            for h, d in zip(host_in, slot_in[slot]):
                if h is not None:
                    d.copy_(h, non_blocking=True)
            in_ready[slot].record(s_in)
        main.wait_event(in_ready[slot])
        if used[slot]:
            main.wait_event(out_free[slot])
        compute(slot)
        done[slot].record(main)
        s_out.wait_event(done[slot])
        with torch.cuda.stream(s_out):
            for h, d in zip(host_out, slot_out[slot]):
                h.copy_(d, non_blocking=True)
            out_free[slot].record(s_out)
        used[slot] = True

    for i in range(warmup):
        step(i)
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(main)
    s_in.wait_stream(main)
    s_out.wait_stream(main)
    for i in range(warmup, warmup + reps):
        step(i)
    main.wait_stream(s_out)
    t1.record(main)
    barrier()
    return t0.elapsed_time(t1) / reps


def cusparse_forward(rp, ci, vals, A, B, S, r, fused_out, timed):
    """FusedMMA by library calls for comparison: the cuSPARSE SDDMM and SpMM
    behind torch.sparse (sampled_addmm, then the values scaled by s, then a
    CSR x dense product), timed like the fused call, checked against it."""
    import torch
    if A.dtype != torch.float32:
        return {"unavailable": "library SDDMM is run for float32 inputs only"}
    try:
        ones = torch.ones(S.nnz, device=A.device) if vals is None else vals
        zero = torch.sparse_csr_tensor(rp, ci, torch.zeros_like(ones), size=(S.m, S.n))
        Bt = B.t()

        def step():
            d = torch.sparse.sampled_addmm(zero, A, Bt, beta=0.0, alpha=1.0)
            v = torch.sparse_csr_tensor(d.crow_indices(), d.col_indices(),
                                        d.values() * ones, size=(S.m, S.n))
            return torch.sparse.mm(v, B)

        got = step()
        rel = float((got - fused_out).norm() / fused_out.norm().clamp_min(1e-30))
        ms = timed(step)
        return {"what": "torch.sparse.sampled_addmm (cuSPARSE SDDMM) + values * s + "
                        "torch.sparse.mm (cuSPARSE SpMM), FusedMMA only",
                "ms": ms, "rel_diff_vs_fused": rel}
    except Exception as ex:  # a library without these CUDA kernels
        return {"unavailable": f"{type(ex).__name__}: {str(ex).splitlines()[0][:160]}"}


def l2_cache_bytes():
    """The L2 size of the current CUDA device (queried), else GB300's 126 MiB."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size)
    except Exception:
        pass
    return 126 << 20


def workload_config(w, args):
    S = w["S"]
    step = ("FusedMMA forward + backward (dA, dB, ds); units = nnz*r per step"
            if args.workload == 3 else "FusedMMA + FusedMMB; units = 2*nnz*r per step")
    e = 4 if w["dtype"] == "f32" else 2
    l2 = l2_cache_bytes()
    dense = (S.m + S.n) * w["r"] * e
    return {"workload": w["name"], "m": S.m, "n": S.n, "nnz": S.nnz, "r": w["r"],
            "input_dtype": w["dtype"], "step": step,
            "l2": ("not flushed: A and B are larger than L2" if dense > 2 * l2
                   else "L2-resident inputs"),
            "parallelism": f"replicas x{args.gpus}", "scale_rows": args.scale}


# ------------------------------------------------------------------ GPU leg

def run_fmm(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2203_07673_gb300 import fmm

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, args.scale, args.bf16)
    S, r, k = w["S"], w["r"], args.workload
    tdt = torch.float32 if w["dtype"] == "f32" else torch.bfloat16
    e = 4 if w["dtype"] == "f32" else 2
    rp = torch.from_numpy(S.row_ptr).to(dev)
    ci = torch.from_numpy(S.col_idx).to(dev)
    if k == 3:
        # s = 1: vals = NULL, the library's every-value-is-one, which still
        # gives the gradient with respect to the values (ds)
        vals = None
    else:
        vals = None if w["vals"] is None else torch.from_numpy(w["vals"]).to(dev)
    A = torch.from_numpy(w["A"]).to(dev).to(tdt).contiguous()
    B = torch.from_numpy(w["B"]).to(dev).to(tdt).contiguous()
    plan = fmm.Plan(rp, ci, S.n, r, tdt)
    info = plan.info()
    out = torch.empty(S.m, r, device=dev)
    out_t = torch.empty(S.n, r, device=dev)
    v = torch.empty(S.nnz, device=dev)
    G = None
    if k == 3:
        G = torch.from_numpy(w["A"].astype(np.float32)).to(dev)   # a fixed upstream gradient
        dA = torch.empty(S.m, r, device=dev)
        dB = torch.empty(S.n, r, device=dev)
        ds = torch.empty(S.nnz, device=dev)
    stream = torch.cuda.current_stream()
    lib = fmm.lib()
    sp = stream.cuda_stream

    def call_fwd():
        fmm.fusedmm(plan, vals, A, B, out=out)

    def call_second():
        if k == 3:
            rc = lib.fmm_fusedmm_bwd(plan.handle, None if vals is None else vals.data_ptr(),
                                     A.data_ptr(), B.data_ptr(), G.data_ptr(), dA.data_ptr(),
                                     dB.data_ptr(), ds.data_ptr(), sp)
            fmm._check(rc, "fmm_fusedmm_bwd")
        else:
            fmm.fusedmm_t(plan, vals, A, B, out=out_t)

    calls = step_calls(k, S, r, e, vals is not None)
    calls_comp = step_calls(k, S, r, e, vals is not None, compulsory_model_bytes)
    fns = [call_fwd, call_second]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        for f in fns:
            f()
    barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(K)]
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for kk in range(K):
        ev[kk][0].record(stream)
        for c, f in enumerate(fns):
            f()
            ev[kk][c + 1].record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    call_ms = [float(np.mean([ev[kk][c].elapsed_time(ev[kk][c + 1]) for kk in range(K)]))
               for c in range(len(fns))]
    elapsed_ms = reduce_max([elapsed_ms], dev, world)[0]

    # unfused path on the same inputs (SDDMM writes v, SpMM reads it back)
    def unfused():
        fmm.sddmm(plan, vals, A, B, out=v)
        fmm.spmm(plan, v, B, out=out)
        if k != 3:
            fmm.sddmm(plan, vals, A, B, out=v)
            fmm.spmm_t(plan, v, A, out=out_t)

    def fused_only():
        fmm.fusedmm(plan, vals, A, B, out=out)
        if k != 3:
            fmm.fusedmm_t(plan, vals, A, B, out=out_t)

    def timed(fn, reps):
        for _ in range(max(3, min(args.warmup, 5))):
            fn()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        barrier()
        return a0.elapsed_time(a1) / reps

    reps = max(3, min(K, 50))
    unfused_ms = timed(unfused, reps)
    fused_ms = timed(fused_only, reps)

    # end to end through the public API from pinned host buffers
    A_h = torch.from_numpy(w["A"]).to(tdt).pin_memory()
    B_h = torch.from_numpy(w["B"]).to(tdt).pin_memory()
    vals_h = None if vals is None else vals.cpu().pin_memory()
    out_h = torch.empty(S.m, r).pin_memory()
    second_h = torch.empty(S.n, r).pin_memory()
    G_h = None if G is None else G.cpu().pin_memory()
    dA_h = None if G is None else torch.empty(S.m, r).pin_memory()
    ds_h = None if G is None else torch.empty(S.nnz).pin_memory()

    # two device copies of every input and output: step i uses slot i % 2,
    # so its uploads overlap step i - 1's compute and read-back
    def second(t):
        return None if t is None else torch.empty_like(t)

    slot_in = [[A, B, vals, G], [second(A), second(B), second(vals), second(G)]]
    outs0 = [out, dB if k == 3 else out_t] + ([dA, ds] if k == 3 else [])
    slot_out = [outs0, [second(t) for t in outs0]]
    host_in = [A_h, B_h, vals_h, G_h]
    host_out = [out_h, second_h] + ([dA_h, ds_h] if k == 3 else [])

    def compute(slot):
        Ab, Bb, vb, Gb = slot_in[slot]
        o = slot_out[slot]
        fmm.fusedmm(plan, vb, Ab, Bb, out=o[0])
        if k == 3:
            rc = lib.fmm_fusedmm_bwd(plan.handle, None if vb is None else vb.data_ptr(),
                                     Ab.data_ptr(), Bb.data_ptr(),
                                     Gb.data_ptr(), o[2].data_ptr(), o[1].data_ptr(),
                                     o[3].data_ptr(), torch.cuda.current_stream().cuda_stream)
            fmm._check(rc, "fmm_fusedmm_bwd")
        else:
            fmm.fusedmm_t(plan, vb, Ab, Bb, out=o[1])

    e2e_reps = max(3, min(K, 30))
    e2e_ms = pipelined_e2e(compute, host_in, slot_in, host_out, slot_out, e2e_reps,
                           max(3, min(args.warmup, 5)), barrier)
    e2e_serial_ms = timed(lambda: serial_e2e(compute, host_in, slot_in, host_out, slot_out),
                          max(3, min(K, 10)))
    library_fwd = None if args.no_library else cusparse_forward(
        rp, ci, vals, A, B, S, r, out, lambda fn: timed(fn, max(3, min(K, 20))))
    unfused_ms, fused_ms, e2e_ms = reduce_max([unfused_ms, fused_ms, e2e_ms], dev, world)

    units_step = (1.0 if k == 3 else 2.0) * S.nnz * r
    value = whole_job_value(units_step, K, world, elapsed_ms)
    ms_per_step = elapsed_ms / K
    peak, peak_kind = load_peaks()
    dom = int(np.argmax(call_ms))
    dom_name, dom_bytes = calls[dom]
    achieved = dom_bytes / (call_ms[dom] / 1e3) / 1e9
    traffic, traffic_note = read_traffic(w["name"], dom_name, w["dtype"])
    # the value permutation of a pass over S^T: one launch, or two (scatter
    # into windows, gather inside them) above two windows of 2^23 slots
    perm_launches = 0 if vals is None else (2 if S.nnz > 2 * (1 << 23) else 1)
    launches = {"fmm_fusedmm": 1 + (1 if info["split_rows"] else 0),
                "fmm_fusedmm_t": 1 + (1 if info["split_cols"] else 0) + perm_launches,
                "fmm_fusedmm_bwd": 2 + (1 if info["split_rows"] else 0)
                + (1 if info["split_cols"] else 0) + perm_launches}
    h2d = A_h.numel() * A_h.element_size() + B_h.numel() * B_h.element_size() + (
        0 if vals_h is None else vals_h.numel() * 4) + (0 if G_h is None else G_h.numel() * 4)
    d2h = (out_h.numel() + second_h.numel()) * 4 + (
        0 if G is None else (dA_h.numel() + ds_h.numel()) * 4)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, args),
        "roofline": {
            "bound": "hbm", "kernel": dom_name,
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_call": dom_bytes,
            "bytes_model": "gather model: CSR + local rows once + one dense row per nonzero "
                           "+ float32 outputs once (+ value permutation on the S^T side)",
            "call_ms": call_ms[dom],
            "dram_frac": None if traffic is None else traffic / (call_ms[dom] / 1e3) / 1e9 / peak,
            "traffic_note": traffic_note,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "nominal_peak": NOMINAL_HBM_GBS,
            "compulsory_bytes_per_call": calls_comp[dom][1],
            "compulsory_frac": calls_comp[dom][1] / (call_ms[dom] / 1e3) / 1e9 / peak,
        },
        "calls": {name: {"ms": call_ms[c], "model_bytes": b,
                         "model_GBs": b / (call_ms[c] / 1e3) / 1e9,
                         "compulsory_bytes": calls_comp[c][1]}
                  for c, (name, b) in enumerate(calls)},
        "library_unfused": library_fwd,
        "fused_vs_unfused": None if k == 3 else {
            "fused_ms": fused_ms, "unfused_ms": unfused_ms,
            "speedup": unfused_ms / fused_ms,
            "unfused": "fmm_sddmm + fmm_spmm + fmm_sddmm + fmm_spmm_t"},
        "e2e": {"value": units_step * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "pipeline": "two buffer sets: uploads on one stream, read-backs on another, "
                            "overlapping the neighbouring steps' compute",
                "serial_ms_per_step": e2e_serial_ms},
        "gpu_launches": K * sum(launches[name] for name, _ in calls),
        "clocks": clk,
        "plan": {kk: info[kk] for kk in ("max_row_nnz", "max_col_nnz", "split_rows",
                                         "split_cols", "variant", "variant_t",
                                         "workspace_bytes")},
    }
    if k == 3:
        line["fused_vs_unfused"] = {"fused_fwd_ms": fused_ms, "unfused_fwd_ms": unfused_ms,
                                    "speedup": unfused_ms / fused_ms,
                                    "unfused": "fmm_sddmm + fmm_spmm"}
    if w["dtype"] == "bf16":
        line["dtype"] = "f32 (bf16 inputs)"
    if k == 2 and not args.no_zipf:
        line["c4"] = zipf_section(args, dev, stream)
    if rank == 0 and not args.no_cpu_baseline:
        cv, desc, threads, _ = oracle_sample(w, args.cpu_seconds)
        line["cpu_baseline"] = {"value": cv, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": desc}
        line["cpu_baseline"].update(single_thread_oracle(w, args.cpu_seconds / 4))
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def zipf_section(args, dev, stream):
    """The Zipf-row workload (2^21 x 2^19, 80M nonzeros, r = 64), drawn on
    the device, in float32 and with bfloat16 A and B: FusedMMA and FusedMMB
    (with the per-call value permutation, and with registered values, i.e.
    the pass alone) timed with CUDA events, each pass beside the gather probe
    on its own index stream (the rows it fetches, in its order, from the same
    table: B for FusedMMA, A in S^T order for FusedMMB)."""
    import torch

    from paper_2203_07673_gb300 import fmm
    from paper_2203_07673_gb300 import workloads as wl

    w = wl.zipf_workload_torch(dev, scale_rows=args.scale)
    rp, ci, vals = w["row_ptr"], w["col_idx"], w["vals"]
    m, n, r, nnz = w["m"], w["n"], w["r"], ci.numel()
    deg = (rp[1:] - rp[:-1]).long()
    rows_t = torch.repeat_interleave(torch.arange(m, device=dev, dtype=torch.int32), deg)
    rows_t = rows_t[torch.argsort(ci, stable=True)].contiguous()
    peak, _ = load_peaks()
    reps = max(5, min(args.steps, 20))

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    res = {"workload": w["name"], "m": m, "n": n, "nnz": nnz, "r": r,
           "max_row_nnz": int(deg.max()), "reps": reps,
           "note": "l2_gather_frac = probe time / pass time: the pass's gather rate as a "
                   "fraction of the rate the same index stream reaches with no arithmetic "
                   "(B, 128 / 64 MiB, mostly L2-resident); gather_ceiling_frac_t the same for "
                   "the FusedMMB pass (A in S^T order, 512 / 256 MiB)"}
    for key, tdt, e in (("fp32", torch.float32, 4), ("bf16", torch.bfloat16, 2)):
        A = w["A"].to(tdt).contiguous()
        B = w["B"].to(tdt).contiguous()
        plan = fmm.Plan(rp, ci, n, r, tdt)
        o = torch.empty(m, r, device=dev)
        ot = torch.empty(n, r, device=dev)
        t_f = timed(lambda: fmm.fusedmm(plan, vals, A, B, out=o))
        t_t = timed(lambda: fmm.fusedmm_t(plan, vals, A, B, out=ot))
        plan.set_values(vals)
        t_tr = timed(lambda: fmm.fusedmm_t(plan, vals, A, B, out=ot))
        plan.set_values(None)
        p_f = timed(lambda: fmm.probe_gather(B, ci))
        p_t = timed(lambda: fmm.probe_gather(A, rows_t))
        model_f = gather_model_bytes(m, nnz, r, e, True)
        model_t = gather_model_bytes(n, nnz, r, e, True)
        name = w["name"] + (" [BF16 A,B]" if key == "bf16" else "")
        tr_f, _ = read_traffic(name, "fmm_fusedmm", key.replace("fp", "f"))
        tr_t, _ = read_traffic(name, "fmm_fusedmm_t", key.replace("fp", "f"))
        info = plan.info()
        res[key] = {
            "fused_ms": t_f, "fused_t_ms": t_t, "fused_t_registered_values_ms": t_tr,
            "permute_ms": t_t - t_tr,
            "gathered_GBs": nnz * r * e / (t_f / 1e3) / 1e9,
            "gathered_GBs_t": nnz * r * e / (t_tr / 1e3) / 1e9,
            "model_frac": model_f / (t_f / 1e3) / 1e9 / peak,
            "model_frac_t": model_t / (t_tr / 1e3) / 1e9 / peak,
            "probe_ms": p_f, "probe_GBs": nnz * r * e / (p_f / 1e3) / 1e9,
            "probe_t_ms": p_t, "probe_t_GBs": nnz * r * e / (p_t / 1e3) / 1e9,
            "l2_gather_frac": p_f / t_f, "gather_ceiling_frac_t": p_t / t_tr,
            "dram_frac": None if tr_f is None else tr_f / (t_f / 1e3) / 1e9 / peak,
            "dram_frac_t": None if tr_t is None else tr_t / (t_t / 1e3) / 1e9 / peak,
            "variant": info["variant"], "variant_t": info["variant_t"],
            "split_nnz": info["split_nnz"],
        }
        plan.close()
        del A, B, o, ot
    return res


def run_dist15d(args, rank, world, local_rank):
    """1.5D dense-shifting FusedMM with local kernel fusion (Algorithm 1)
    over the ranks, replication factor --dist-c, weak-scaled like the
    paper's Erdos-Renyi setup: each rank owns 2^20 rows (times --scale) of
    an ER pattern with 32 distinct uniform columns per row over all
    N x 2^20 columns, r = 128, FP32, s ~ U(0,1), A, B ~ N(0, 1/128), drawn
    on its device.  A step is FusedMMA + FusedMMB over the whole matrix
    (N / c phases each); units 2 * nnz * r of the whole matrix per step."""
    import torch
    import torch.distributed as dist

    from paper_2203_07673_gb300 import dist15d
    from paper_2203_07673_gb300 import workloads as wl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rows = max(1, int((1 << 20) * args.scale))
    n = rows * world
    r = 128
    c = args.dist_c
    if c < 1 or world % c:
        raise SystemExit(f"--dist-c {c} must divide the {world} ranks")
    lp = world // c
    layer, q = divmod(rank, lp)
    bounds = [l * rows for l in range(world + 1)]
    # the fiber's c row blocks are drawn alike by its c ranks (one seed per
    # fiber); each keeps the columns of its layer's B blocks
    g = wl._torch_gen(dev, (wl.ROOT_SEED + 2) * 1000003 + 15 + q)
    rp_f, ci_f = wl.er_exact_degree_torch(c * rows, n, 32, g, dev)
    vals_f = torch.rand(ci_f.numel(), generator=g, device=dev)
    rp, ci, slots = dist15d.local_block(rp_f, ci_f, 0, c * rows, bounds[layer * lp],
                                        bounds[(layer + 1) * lp])
    vals = vals_f.index_select(0, slots)
    del rp_f, ci_f, vals_f, slots
    g = wl._torch_gen(dev, (wl.ROOT_SEED + 2) * 1000003 + 7919 + rank)
    A = torch.randn(rows, r, generator=g, device=dev) * (1.0 / 128) ** 0.5
    B = torch.randn(rows, r, generator=g, device=dev) * (1.0 / 128) ** 0.5
    d = dist15d.FusedMM15D(rp, ci, n, r, torch.float32, col_bounds=bounds, c=c,
                           row_bounds=bounds)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step(vk, Ak, Bk):
        return d.fusedmm(vk, Ak, Bk), d.fusedmm_t(vk, Ak, Bk)

    for _ in range(args.warmup):
        step(vals, A, B)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for _ in range(args.steps):
        step(vals, A, B)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed = reduce_max([t0.elapsed_time(t1)], dev, world)[0]
    # end to end: every step uploads this rank's A, B and values from pinned
    # host memory and reads both output blocks back
    A_h, B_h, v_h = A.cpu().pin_memory(), B.cpu().pin_memory(), vals.cpu().pin_memory()
    o_h = torch.empty((rows, r), dtype=torch.float32).pin_memory()
    ot_h = torch.empty((rows, r), dtype=torch.float32).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(reps):
        o, ot = step(v_h.to(dev, non_blocking=True), A_h.to(dev, non_blocking=True),
                     B_h.to(dev, non_blocking=True))
        o_h.copy_(o, non_blocking=True)
        ot_h.copy_(ot, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = reduce_max([e0.elapsed_time(e1) / reps], dev, world)[0]
    h2d_local = (A_h.numel() + B_h.numel() + v_h.numel()) * 4
    if world > 1:
        t = torch.tensor([float(h2d_local)], device=dev, dtype=torch.float64)
        dist.all_reduce(t)
        h2d_total = int(t.item())
    else:
        h2d_total = h2d_local
    nnz_total = 32 * rows * world   # every row of S holds 32 nonzeros
    units = 2.0 * nnz_total * r
    # library launches per step: per phase one FusedMMA pass (+ its combine
    # where rows are split) and one FusedMMB pass (+ combine) after the value
    # permutation (one launch, or two above two windows of 2^23 slots)
    per_step = 0
    for pl in d.plans:
        info = pl.info()
        nnz_l = int(info.get("nnz", 0))
        per_step += 1 + (1 if info["split_rows"] else 0)
        per_step += 1 + (1 if info["split_cols"] else 0) + (2 if nnz_l > 2 * (1 << 23) else 1)
    d.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": whole_job_value(units / world, args.steps, world, elapsed),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"1.5D dense shifting + local kernel fusion (Algorithm 1, "
                                   f"c = {c}): ER {n}x{n}, 32 nnz/row, r=128, FP32, {rows} rows "
                                   f"per rank",
                       "m": n, "n": n, "nnz": nnz_total, "r": r,
                       "step": "FusedMMA + FusedMMB over the whole matrix",
                       "parallelism": f"1.5D grid {lp}x{c}"},
            "e2e": {"value": units / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d_total,
                    "d2h_bytes_per_step": 2 * rows * r * 4 * world, "ms_per_step": e2e_ms},
            "gpu_launches": per_step * args.steps, "clocks": clk}), flush=True)
    return 0


def run_batched(args, rank, world, local_rank):
    """Workload 5: 512 uneven matrices, BF16 inputs, forward + backward as one
    persistent launch each (fmm_batch_forward / fmm_batch_backward), replayed
    from CUDA graphs; variants picked by the autotuner per shape group."""
    import torch
    import torch.distributed as dist

    from paper_2203_07673_gb300 import autotune, fmm
    from paper_2203_07673_gb300 import workloads as wl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    specs = wl.batched_specs(args.batch_count, scale_rows=args.scale)
    t0 = time.perf_counter()
    items, mats = [], []
    for t, sp in enumerate(specs):
        m = wl.batched_matrix_torch(sp, t, dev)
        r = m["r"]
        plan = fmm.Plan(m["row_ptr"], m["col_idx"], m["n"], r, torch.bfloat16,
                        split_nnz=1 << 30)
        g = torch.Generator(device=dev)
        g.manual_seed(7919 * t + 1)
        items.append(dict(plan=plan, vals=m["vals"], A=m["A"].bfloat16().contiguous(),
                          B=m["B"].bfloat16().contiguous(),
                          G=torch.randn(m["m"], r, device=dev, generator=g),
                          out=torch.empty(m["m"], r, device=dev),
                          dA=torch.empty(m["m"], r, device=dev),
                          dB=torch.empty(m["n"], r, device=dev),
                          ds=torch.empty(m["col_idx"].numel(), device=dev),
                          rp=m["row_ptr"], ci=m["col_idx"]))
        mats.append(m)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tuned = autotune.tune_batch(items) if not args.no_tune else {}
    tune_s = time.perf_counter() - t0
    keys = ("plan", "vals", "A", "B", "out", "G", "dA", "dB", "ds")
    batch = fmm.Batch([{k: it[k] for k in keys} for it in items])
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.forward(); batch.backward()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g_fwd, g_bwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_fwd):
        batch.forward()
    with torch.cuda.graph(g_bwd):
        batch.backward()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        g_fwd.replay(); g_bwd.replay()
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    barrier()
    t_s = torch.cuda.Event(enable_timing=True); t_e = torch.cuda.Event(enable_timing=True)
    t_s.record(stream)
    for kk in range(K):
        ev[kk][0].record(stream)
        g_fwd.replay()
        ev[kk][1].record(stream)
        g_bwd.replay()
        ev[kk][2].record(stream)
    t_e.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t_s.elapsed_time(t_e)
    fwd_ms = float(np.mean([ev[kk][0].elapsed_time(ev[kk][1]) for kk in range(K)]))
    bwd_ms = float(np.mean([ev[kk][1].elapsed_time(ev[kk][2]) for kk in range(K)]))
    elapsed_ms = reduce_max([elapsed_ms], dev, world)[0]

    def timed(fn, reps=3):
        fn()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        barrier()
        return a0.elapsed_time(a1) / reps

    v_bufs = [torch.empty(it["ci"].numel(), device=dev) for it in items]
    # the per-matrix baselines use plans of their own with the library's
    # defaults (variant and long-row splitting: the batch's plans split no
    # rows, which one matrix at a time would leave hub rows on one team)
    base_plans = [fmm.Plan(it["rp"], it["ci"], it["plan"].n, it["plan"].r, torch.bfloat16)
                  for it in items]

    def per_matrix_fused():
        for it, bp in zip(items, base_plans):
            fmm.fusedmm(bp, it["vals"], it["A"], it["B"], out=it["out"])

    def per_matrix_unfused():
        for it, bp, v in zip(items, base_plans, v_bufs):
            fmm.sddmm(bp, it["vals"], it["A"], it["B"], out=v)
            fmm.spmm(bp, v, it["B"], out=it["out"])

    # the per-matrix baselines replay from CUDA graphs too, so both sides of
    # the comparison are GPU time (512 launches from Python would measure
    # the host)
    def graphed(fn):
        side_s = torch.cuda.Stream()
        side_s.wait_stream(stream)
        with torch.cuda.stream(side_s):
            fn()
        stream.wait_stream(side_s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            fn()
        return graph

    g_pm_fused, g_pm_unfused = graphed(per_matrix_fused), graphed(per_matrix_unfused)
    loop_fused_ms = timed(g_pm_fused.replay)
    loop_unfused_ms = timed(g_pm_unfused.replay)

    # end to end: inputs from pinned host memory, outputs back, every step
    host_in = [(it[k].cpu().pin_memory(), it[k]) for it in items for k in ("vals", "A", "B", "G")]
    host_out = [(torch.empty(it[k].shape).pin_memory(), it[k]) for it in items
                for k in ("out", "dA", "dB", "ds")]

    def e2e_step():
        for h, d in host_in:
            d.copy_(h, non_blocking=True)
        g_fwd.replay(); g_bwd.replay()
        for h, d in host_out:
            h.copy_(d, non_blocking=True)

    e2e_ms = timed(e2e_step, 2)
    h2d = sum(h.numel() * h.element_size() for h, _ in host_in)
    d2h = sum(h.numel() * h.element_size() for h, _ in host_out)

    nnz = [it["ci"].numel() for it in items]
    rs = [it["plan"].r for it in items]
    units_step = float(sum(z * r for z, r in zip(nnz, rs)))
    value = whole_job_value(units_step, K, world, elapsed_ms)
    fwd_bytes = sum(gather_model_bytes(it["plan"].m, z, r, 2, True) for it, z, r in zip(items, nnz, rs))
    bwd_bytes = sum(gather_model_bytes(it["plan"].m, z, r, 2, True) + 4 * it["plan"].m * r + 4 * z
                    + gather_model_bytes(it["plan"].n, z, r, 2, True) + 4 * z * r + 4 * z
                    for it, z, r in zip(items, nnz, rs))
    peak, peak_kind = load_peaks()
    dom_ms, dom_bytes, dom_name = (bwd_ms, bwd_bytes, "batch_kernel<bf16, backward>") \
        if bwd_ms >= fwd_ms else (fwd_ms, fwd_bytes, "batch_kernel<bf16, forward>")
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 inputs)",
        "data": "synthetic",
        "config": {"workload": wl.WORKLOADS[5], "matrices": len(items), "rows": int(sum(
            it["plan"].m for it in items)), "nnz": int(sum(nnz)), "r_mix": {
            str(r): rs.count(r) for r in (32, 64, 128)},
            "step": "batched FusedMMA forward + backward (dA, dB, ds), one persistent launch "
                    "each, replayed from CUDA graphs; units = sum nnz*r per step",
            "l2": "not flushed: the batch's operands total several GB",
            "parallelism": f"replicas x{args.gpus}", "scale_rows": args.scale},
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_call": dom_bytes, "call_ms": dom_ms,
                     "bytes_model": "gather model summed over the matrices"},
        "calls": {"batch_forward": {"ms": fwd_ms, "model_bytes": fwd_bytes,
                                    "model_GBs": fwd_bytes / (fwd_ms / 1e3) / 1e9},
                  "batch_backward": {"ms": bwd_ms, "model_bytes": bwd_bytes,
                                     "model_GBs": bwd_bytes / (bwd_ms / 1e3) / 1e9}},
        "batching": {"per_matrix_fused_forward_ms": loop_fused_ms,
                     "per_matrix_unfused_forward_ms": loop_unfused_ms,
                     "batched_forward_ms": fwd_ms,
                     "speedup_vs_per_matrix_fused": loop_fused_ms / fwd_ms,
                     "speedup_vs_per_matrix_unfused": loop_unfused_ms / fwd_ms,
                     "per_matrix": "512 fused (1024 unfused) launches replayed from CUDA graphs, "
                                   "plans with the library defaults (variant, long-row split)"},
        "e2e": {"value": units_step * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": 2 * K,
        "clocks": clk,
        "setup": {"generate_s": gen_s, "autotune_s": tune_s, "tuned_groups": len(tuned),
                  "tuned_codes": tuned},
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        done_units, t_cpu, used = 0.0, 0.0, 0
        for it, m in zip(items, mats):
            if t_cpu >= args.cpu_seconds:
                break
            rp = m["row_ptr"].cpu().numpy(); ci = m["col_idx"].cpu().numpy()
            a = it["A"].double().cpu().numpy(); b = it["B"].double().cpu().numpy()
            v = m["vals"].double().cpu().numpy(); g_ = it["G"].double().cpu().numpy()
            c0 = time.perf_counter()
            oracle.fusedmm(rp, ci, v, a, b, m["n"])
            oracle.fusedmm_grad(rp, ci, v, a, b, g_, m["n"])
            t_cpu += time.perf_counter() - c0
            done_units += ci.size * m["r"]
            used += 1
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = {
            "value": done_units / t_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {used} of {len(items)} matrices, FusedMMA (rows on {threads} "
                      "OpenMP threads) + its gradient (sequential) in FP64 on the BF16-rounded "
                      "inputs (oracle/fmm_oracle.c)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    for it in items:
        it["plan"].close()
    return 0


def run_als(args, rank, world, local_rank):
    """ALS with batched CG (Sec. VI-E) on the workload-4 pattern: one sweep
    = `--cg-iters` CG iterations for A then as many for B; every CG query is
    one FusedMM over the 0/1 pattern, every CG step's row work one kernel."""
    import torch

    from paper_2203_07673_gb300 import als, fmm

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(4, args.scale)
    S, r = w["S"], w["r"]
    rp = torch.from_numpy(S.row_ptr).to(dev)
    ci = torch.from_numpy(S.col_idx).to(dev)
    c = torch.from_numpy(w["vals"]).to(dev)
    A0 = torch.from_numpy(w["A"]).to(dev)
    B0 = torch.from_numpy(w["B"]).to(dev)
    plan = fmm.Plan(rp, ci, S.n, r)
    A, B = A0.clone(), B0.clone()
    lam, iters = args.als_lambda, args.cg_iters
    solver = als.ALS(plan, c, A, B, lam)
    loss0 = solver.loss()
    for _ in range(max(3, args.warmup)):
        solver.sweep(iters)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    stream = torch.cuda.current_stream()
    K = args.steps
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        solver.sweep(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sweep_ms = e0.elapsed_time(e1) / K
    loss1 = solver.loss()

    # breakdown: the FusedMM queries and the CG row updates of one A side
    q = torch.empty(S.m, r, device=dev)
    res = torch.empty(S.m, r, device=dev); p = torch.empty(S.m, r, device=dev)
    rs = torch.ones(S.m, device=dev)

    def time_of(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    p.copy_(A)
    t_query_a = time_of(lambda: fmm.fusedmm(plan, None, p, B, out=q))
    t_update_a = time_of(lambda: fmm.cg_update(lam, A, res, p, q, rs))
    qn = torch.empty(S.n, r, device=dev); pn = B.clone()
    t_query_b = time_of(lambda: fmm.fusedmm_t(plan, None, A, pn, out=qn))
    fused_calls = 2 * (iters + 1)
    units_sweep = fused_calls * float(S.nnz) * r

    # end to end: c, A and B from pinned host memory, one sweep, the factors
    # read back
    c_h, A_h, B_h = c.cpu().pin_memory(), A0.cpu().pin_memory(), B0.cpu().pin_memory()
    Ao_h, Bo_h = torch.empty_like(A_h).pin_memory(), torch.empty_like(B_h).pin_memory()

    def e2e_step():
        c.copy_(c_h, non_blocking=True)
        A.copy_(A_h, non_blocking=True)
        B.copy_(B_h, non_blocking=True)
        solver.sweep(iters)
        Ao_h.copy_(A, non_blocking=True)
        Bo_h.copy_(B, non_blocking=True)

    e2e_ms = time_of(e2e_step, max(3, K))
    h2d = (c_h.numel() + A_h.numel() + B_h.numel()) * 4
    d2h = (Ao_h.numel() + Bo_h.numel()) * 4
    peak, peak_kind = load_peaks()
    q_bytes = gather_model_bytes(S.m, S.nnz, r, 4, vals=False)
    traffic, traffic_note = read_traffic(w["name"], "fmm_fusedmm (pattern only)", "f32")
    line = {
        "metric": METRIC, "value": units_sweep / (sweep_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": K, "warmup": args.warmup, "ms_per_step": sweep_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ALS with CG on " + w["name"], "m": S.m, "n": S.n,
                   "nnz": S.nnz, "r": r, "lambda": lam, "cg_iters_per_side": iters,
                   "step": f"one ALS sweep: {iters} CG iterations for A, then {iters} for B; "
                           f"units = nnz*r per FusedMM query ({fused_calls} per sweep)"},
        "als": {"loss_before": loss0, "loss_after": loss1,
                "fusedmm_query_ms_A": t_query_a, "fusedmm_query_ms_B": t_query_b,
                "cg_row_update_ms_A": t_update_a,
                "row_update_share": iters * t_update_a / (sweep_ms / 2)},
        "roofline": {"bound": "hbm", "kernel": "fmm_fusedmm (CG query M p, pattern only)",
                     "achieved": q_bytes / (t_query_a / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": q_bytes / (t_query_a / 1e3) / 1e9 / peak, "traffic": traffic,
                     "traffic_note": traffic_note,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_call": q_bytes, "call_ms": t_query_a,
                     "bytes_model": "gather model without values: CSR + local rows once + one "
                                    "dense row per nonzero + float32 output once"},
        "e2e": {"value": units_sweep / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        # per side: b (SpMM), M x0, cg_init, then per iteration a query and a
        # row update; the B side's SpMM^T first permutes c; split rows add
        # a combine per pass over S
        "gpu_launches": K * (2 * (3 + 2 * iters) + 1 + (
            (2 + iters) if plan.info()["split_rows"] else 0) + (
            (2 + iters) if plan.info()["split_cols"] else 0)),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        import oracle
        rows = max(256, int(S.m * 0.004))
        sub = S.rows_slice(0, rows)
        cols, ci_s = np.unique(sub.col_idx, return_inverse=True)
        a = w["A"][:rows].astype(np.float64); b = w["B"][cols].astype(np.float64)
        cv = w["vals"][:sub.nnz].astype(np.float64)
        t0 = time.perf_counter()
        oracle.als_cg(sub.row_ptr, ci_s.astype(np.int64), cv, a, b, lam, iters, 0)
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {
            "value": (iters + 1) * sub.nnz * r / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"A-side CG ({iters} iterations) of the first {rows} rows ({sub.nnz} nnz) "
                      "in FP64, sequential (oracle/fmm_oracle.c)"}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_probe(args, dev):
    """Gather ceilings (fmm_probe_gather): the rate at which a stream of
    uniform random row indices fetches rows of a table and nothing else,
    for tables from L2-resident to far beyond L2, rows of 128 and 256 bytes
    (BF16 and FP32 rows of r = 64), 80M indices (the Zipf-row workload's
    nonzero count), CUDA events over 10 launches after 3 warm-ups."""
    import torch

    from paper_2203_07673_gb300 import fmm

    count = int(80_000_000 * args.scale)
    g = torch.Generator(device=dev)
    g.manual_seed(2203_07673)
    rows_out = []
    for mib in (32, 64, 128, 512, 2048):
        for row_bytes in (128, 256):
            rows = (mib << 20) // row_bytes
            table = torch.randn(rows, row_bytes // 4, device=dev, generator=g)
            idx = torch.randint(0, rows, (count,), device=dev, dtype=torch.int32, generator=g)
            sink = torch.zeros(1, dtype=torch.int32, device=dev)
            for _ in range(3):
                fmm.probe_gather(table, idx, sink)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                fmm.probe_gather(table, idx, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            rows_out.append({"table_MiB": mib, "row_bytes": row_bytes, "ms": ms,
                             "rows_per_s": count / (ms / 1e3),
                             "gathered_GBs": count * row_bytes / (ms / 1e3) / 1e9})
            del table, idx
    return {"probe": "fmm_probe_gather, uniform random row indices", "indices": count,
            "rows": rows_out}


def run_gat(args, rank, world, local_rank):
    """Graph-attention forward (Sec. VI-E) on an R-MAT 2^22 graph (avg degree
    16, the workload-3 recipe drawn on the device), `--heads` heads of
    `--head-dim` features, random weights as in the paper."""
    import torch

    from paper_2203_07673_gb300 import fmm, gat
    from paper_2203_07673_gb300 import workloads as wl

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    scale = 22
    while scale > 8 and (1 << scale) > (1 << 22) * args.scale:
        scale -= 1
    nv = 1 << scale
    gen = wl._torch_gen(dev, wl.ROOT_SEED + 3)
    rp, ci = wl.rmat_torch(scale, 16 * nv, 0.57, 0.19, 0.19, gen, dev, nv)
    heads, rh = args.heads, args.head_dim
    r = heads * rh
    tdt = torch.bfloat16 if args.gat_bf16 else torch.float32
    plan = fmm.Plan(rp, ci, nv, r, tdt)
    X = torch.randn(nv, r, device=dev, generator=gen)
    W = torch.randn(r, r, device=dev, generator=gen) / r ** 0.5
    a_l = torch.randn(r, device=dev, generator=gen)
    a_r = torch.randn(r, device=dev, generator=gen)
    H = X @ W
    f = fmm.gat_project(H, a_l, heads)
    g = fmm.gat_project(H, a_r, heads)
    Hp = H.to(tdt).contiguous()
    out = torch.empty(nv, r, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    clocks = ClockSampler(local_rank)
    clocks.start()
    attn_ms = timed(lambda: fmm.gat_forward(plan, heads, None, f, g, Hp, 0.2, out=out), args.steps)
    clk = clocks.stop()
    # end to end: H, f and g from pinned host memory, the output read back
    Hh, fh, gh = Hp.cpu().pin_memory(), f.cpu().pin_memory(), g.cpu().pin_memory()
    out_h = torch.empty(nv, r).pin_memory()

    def e2e_step():
        Hp.copy_(Hh, non_blocking=True)
        f.copy_(fh, non_blocking=True)
        g.copy_(gh, non_blocking=True)
        fmm.gat_forward(plan, heads, None, f, g, Hp, 0.2, out=out)
        out_h.copy_(out, non_blocking=True)

    e2e_ms = timed(e2e_step, max(3, args.steps // 2))
    h2d = Hh.numel() * Hh.element_size() + (fh.numel() + gh.numel()) * 4
    d2h = out_h.numel() * 4
    layer_ms = timed(lambda: gat.gat_layer(plan, X, W, a_l, a_r, heads), max(3, args.steps // 4))
    nnz = ci.numel()
    e = 4 if tdt == torch.float32 else 2
    model = 4 * (nv + 1) + 4 * nnz + nnz * (r * e + 4 * heads) + nv * (4 * heads + 4 * r)
    peak, peak_kind = load_peaks()
    wname = (f"GAT forward, R-MAT 2^{scale} (a,b,c,d)=(.57,.19,.19,.05), avg degree 16, "
             f"{heads} heads x {rh}")
    traffic, traffic_note = read_traffic(wname, "fmm_gat_forward", "bf16" if e == 2 else "f32")
    info = plan.info()
    line = {
        "metric": METRIC, "value": nnz * r / (attn_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": attn_ms,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" + (" (bf16 H)" if tdt == torch.bfloat16 else ""), "data": "synthetic",
        "config": {"workload": wname, "nnz": nnz, "r": r, "slope": 0.2,
                   "l2": "not flushed: H is larger than L2",
                   "step": "fmm_gat_forward (scores, row softmax, aggregation); units = nnz*r"},
        "roofline": {"bound": "hbm", "kernel": "gat_kernel", "achieved": model / (attn_ms / 1e3) / 1e9,
                     "peak": peak, "unit": "GB/s",
                     "frac": model / (attn_ms / 1e3) / 1e9 / peak, "traffic": traffic,
                     "dram_frac": None if traffic is None else traffic / (attn_ms / 1e3) / 1e9 / peak,
                     "traffic_note": traffic_note,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "bytes_model": "CSR + one H row and the head scores g_j per nonzero + f_i "
                                    "and the output row per row"},
        "gat": {"attention_ms": attn_ms, "layer_ms": layer_ms,
                "layer": "X W (torch.matmul) + projections + attention"},
        "e2e": {"value": nnz * r / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": args.steps * (1 + (1 if info["split_rows"] else 0)), "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = gat_oracle_sample(rp, ci, f, g, Hp, heads, r, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def gat_oracle_sample(rp, ci, f, g, Hp, heads, r, seconds):
    """The FP64 oracle's attention forward on the first rows of the graph
    (columns remapped to the ones they touch), sized to about `seconds`."""
    import oracle
    rp_h = rp.cpu().numpy().astype(np.int64)
    ci_h = ci.cpu().numpy()
    f_h = f.double().cpu().numpy()
    g_h = g.double().cpu().numpy()

    def run(rows):
        nz = int(rp_h[rows])
        cols, cmap = np.unique(ci_h[:nz], return_inverse=True)
        H = Hp[torch_index(cols, Hp.device)].double().cpu().numpy()
        t0 = time.perf_counter()
        oracle.gat(rp_h[:rows + 1], cmap, None, f_h[:rows], g_h[cols], H, heads, 0.2)
        return time.perf_counter() - t0, nz

    rows = min(len(rp_h) - 1, 4096)
    t, nz = run(rows)
    rows = int(min(len(rp_h) - 1, max(rows, rows * seconds / max(t, 1e-6))))
    t, nz = run(rows)
    return {"value": nz * r / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {rows} rows ({nz} nnz) of the graph, columns remapped to the ones "
                      f"they touch; attention forward in FP64 (oracle/fmm_oracle.c)"}


def torch_index(idx, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(device)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fmm", "reference"], default="fmm")
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--batch-count", type=int, default=512, help="matrices of workload 5")
    ap.add_argument("--no-tune", action="store_true", help="workload 5 without the autotuner")
    ap.add_argument("--als", action="store_true", help="ALS with batched CG on workload 4's pattern")
    ap.add_argument("--als-lambda", type=float, default=0.1)
    ap.add_argument("--cg-iters", type=int, default=10)
    ap.add_argument("--gat", action="store_true", help="graph-attention forward on an R-MAT graph")
    ap.add_argument("--heads", type=int, default=4)
    ap.add_argument("--head-dim", type=int, default=32)
    ap.add_argument("--gat-bf16", action="store_true")
    ap.add_argument("--bf16", action="store_true",
                    help="workloads 2 and 4 with BF16 A and B (FP32 accumulation)")
    ap.add_argument("--scale", type=float, default=1.0, help="row-count scale (1 = full)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clock-log", default=None,
                    help="keep nvidia-smi's raw clock samples under this path prefix")
    ap.add_argument("--no-zipf", action="store_true",
                    help="default workload without the Zipf-row (c4) section")
    ap.add_argument("--dist15d", action="store_true",
                    help="1.5D dense-shifting FusedMM over the ranks (weak-scaled ER, 2^20 rows "
                         "per rank); without it N > 1 runs independent replicas")
    ap.add_argument("--dist-c", type=int, default=1,
                    help="replication factor of --dist15d (divides N)")
    ap.add_argument("--zipf-only", action="store_true",
                    help="only the Zipf-row (c4) section, printed as one JSON object")
    ap.add_argument("--probe", action="store_true",
                    help="gather ceilings of uniform random rows, tables of 32 MiB to 2 GiB")
    ap.add_argument("--no-library", action="store_true",
                    help="skip the cuSPARSE (torch.sparse) comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ClockSampler.log_path = args.clock_log
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
    if args.zipf_only:
        import torch
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        res = zipf_section(args, dev, torch.cuda.current_stream())
        if rank == 0:
            print(json.dumps(res), flush=True)
        rc = 0
    elif args.probe:
        import torch
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        res = run_probe(args, dev)
        if rank == 0:
            print(json.dumps(res), flush=True)
        rc = 0
    elif args.dist15d:
        rc = run_dist15d(args, rank, world, local_rank)
    elif args.als:
        rc = run_als(args, rank, world, local_rank)
    elif args.gat:
        rc = run_gat(args, rank, world, local_rank)
    else:
        rc = (run_batched if args.workload == 5 else run_fmm)(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
