"""Autotuner of the row-pass kernel variants (rows per warp and r-tiling).

A variant code V*100 + N*10 + U fixes how a row pass maps onto the GPU:
V vectors per lane (with the row width, the lanes per dense row, i.e. the
r-tiling), N lane groups sharing one output row (with V, the rows per warp)
and U nonzeros per group per batch; the staged (1xxx), register-ring
(2xxxx, 3xxxx) and streaming (5xxxx) codes keep gathered rows in flight in
shared memory or registers (include/fmm.h lists them).  ``tune_plan`` times
every candidate, and the plan's current codes, on the plan's own operands
with CUDA events and keeps the fastest, separately for the passes over S
and over S^T.  ``tune_batch`` groups the items of a
batch by a signature of their shape (r, dtype, average and largest row
length, as powers of two), tunes one item per group and applies the result
to the group; results can be cached in a JSON file keyed by the signature.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import fmm

ALL_CODES = (112, 114, 118, 122, 124, 212, 214, 221, 222, 224, 441, 442, 1041, 1042, 1081, 1082,
             22212, 22412, 32212, 52412)
BATCH_CODES = (112, 114, 122, 212, 214, 221)


def _time(fn, iters=5, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def signature(plan: fmm.Plan) -> str:
    info = plan.info()
    lg = lambda x: int(math.floor(math.log2(max(1.0, x))))
    avg_r = plan.nnz / max(1, plan.m)
    avg_c = plan.nnz / max(1, plan.n)
    return (f"r{plan.r}-{'bf16' if plan.dtype == torch.bfloat16 else 'f32'}"
            f"-a{lg(avg_r)}-m{lg(info['max_row_nnz'])}"
            f"-ac{lg(avg_c)}-mc{lg(max(1, info['max_col_nnz']))}")


def tune_plan(plan: fmm.Plan, vals, A, B, G=None, candidates=ALL_CODES, iters=5,
              backward=True):
    """Times each candidate on this plan's operands; sets and returns the
    fastest (variant over S, variant over S^T) with the measured times."""
    m, n, r = plan.m, plan.n, plan.r
    out = torch.empty(m, r, device=plan.device)
    out_t = torch.empty(n, r, device=plan.device)
    if backward and G is not None:
        lib, sp = fmm.lib(), torch.cuda.current_stream().cuda_stream
        dA = torch.empty(m, r, device=plan.device)
        dB = torch.empty(n, r, device=plan.device)
        ds = torch.empty(plan.nnz, device=plan.device)
        vp = None if vals is None else vals.data_ptr()

        def s_side():
            fmm.fusedmm(plan, vals, A, B, out=out)
            lib.fmm_fusedmm_bwd(plan.handle, vp, A.data_ptr(), B.data_ptr(), G.data_ptr(),
                                dA.data_ptr(), None, ds.data_ptr(), sp)

        def t_side():
            lib.fmm_fusedmm_bwd(plan.handle, vp, A.data_ptr(), B.data_ptr(), G.data_ptr(),
                                None, dB.data_ptr(), None, sp)
    else:
        def s_side():
            fmm.fusedmm(plan, vals, A, B, out=out)

        def t_side():
            fmm.fusedmm_t(plan, vals, A, B, out=out_t)

    info = plan.info()
    current = (info["variant"], info["variant_t"])
    times_s, times_t = {}, {}
    for code in dict.fromkeys(tuple(candidates) + current):
        plan.set_variant(code, code)
        times_s[code] = _time(s_side, iters)
        times_t[code] = _time(t_side, iters)
    best_s = min(times_s, key=times_s.get)
    best_t = min(times_t, key=times_t.get)
    plan.set_variant(best_s, best_t)
    return {"variant": best_s, "variant_t": best_t, "ms": times_s, "ms_t": times_t}


def tune_batch(items, cache_path: str | None = None, candidates=BATCH_CODES, iters=3,
               min_gain=0.01):
    """Tunes the plans of batch items (dicts with plan, vals, A, B, out and
    optionally G, dA, dB, ds) in the batch's own setting: one persistent
    kernel per phase, whose register count is fixed by its heaviest path, so
    per-plan timings do not carry over.  Items are grouped by row width and
    dtype; for each group in turn every candidate code is set on that
    group's plans (the other groups keep their current codes), the batch is
    rebuilt and its forward + backward timed, and the group keeps the fastest
    code if it beats the current one by more than min_gain.  Returns
    {group: code}."""
    keys = ("plan", "vals", "A", "B", "out", "G", "dA", "dB", "ds")
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = {k: int(v) for k, v in json.load(fh).items()}
    groups = {}
    for it in items:
        p = it["plan"]
        groups.setdefault(f"r{p.r}-{'bf16' if p.dtype == torch.bfloat16 else 'f32'}",
                          []).append(it)
    backward = all(it.get("G") is not None for it in items)

    def batch_ms():
        batch = fmm.Batch([{k: it.get(k) for k in keys} for it in items])
        try:
            def step():
                batch.forward()
                if backward:
                    batch.backward()
            return _time(step, iters)
        finally:
            batch.close()

    for g, members in groups.items():
        if g in cache:
            for it in members:
                it["plan"].set_variant(cache[g], cache[g])
    best = batch_ms()
    for g, members in groups.items():
        if g in cache:
            continue
        current = members[0]["plan"].info()["variant"]
        choice = current
        for code in candidates:
            if code == current:
                continue
            for it in members:
                it["plan"].set_variant(code, code)
            t = batch_ms()
            if t < best * (1.0 - min_gain):
                best, choice = t, code
        for it in members:
            it["plan"].set_variant(choice, choice)
        cache[g] = choice
    if cache_path:
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
    return cache
