"""Host logic of the batch autotuner (CPU): candidates are judged by the
time of the batched launch itself, per row-width group, and a group keeps
its code unless a candidate is faster by more than min_gain."""
import json

import torch

from paper_2203_07673_gb300 import autotune


class FakePlan:
    def __init__(self, r, code=112):
        self.r, self.dtype, self.code = r, torch.bfloat16, code

    def info(self):
        return {"variant": self.code}

    def set_variant(self, v, vt):
        assert v == vt
        self.code = v


def run(monkeypatch, items, cost, **kw):
    """cost(codes by width) -> ms of one batched step."""
    built = []

    class FakeBatch:
        def __init__(self, its):
            self.codes = {it["plan"].r: it["plan"].code for it in its}
            built.append(self.codes)

        def forward(self):
            pass

        def backward(self):
            pass

        def close(self):
            pass

    monkeypatch.setattr(autotune.fmm, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "_time", lambda fn, iters: (fn(), cost(built[-1]))[1])
    return autotune.tune_batch(items, **kw), built


def items_of(*rs):
    return [dict(plan=FakePlan(r), vals=None, A=None, B=None, out=None) for r in rs]


def test_keeps_defaults_when_no_candidate_is_faster(monkeypatch):
    items = items_of(32, 64, 64, 128)
    tuned, built = run(monkeypatch, items, lambda codes: 10.0)
    assert tuned == {"r32-bf16": 112, "r64-bf16": 112, "r128-bf16": 112}
    assert all(it["plan"].code == 112 for it in items)
    # one baseline plus every other candidate once per group
    assert len(built) == 1 + 3 * (len(autotune.BATCH_CODES) - 1)


def test_picks_a_faster_code_per_group_in_the_batch(monkeypatch):
    items = items_of(32, 64, 128)

    def cost(codes):   # 122 helps r = 64 by 5 %, 214 helps r = 128 by 0.5 % (noise)
        t = 10.0
        if codes[64] == 122:
            t -= 0.5
        if codes[128] == 214:
            t -= 0.05
        return t

    tuned, _ = run(monkeypatch, items, cost, min_gain=0.01)
    assert tuned["r64-bf16"] == 122 and tuned["r128-bf16"] == 112 and tuned["r32-bf16"] == 112
    assert [it["plan"].code for it in items] == [112, 122, 112]


def test_cache_round_trip(monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    items = items_of(64)
    tuned, _ = run(monkeypatch, items, lambda c: 9.0 if c[64] == 221 else 10.0,
                   cache_path=str(path))
    assert json.loads(path.read_text()) == {"r64-bf16": 221} == tuned
    # a cached group is applied without a search: only the baseline batch is timed
    fresh = items_of(64)
    calls = []
    tuned2, built = run(monkeypatch, fresh, lambda c: calls.append(dict(c)) or 10.0,
                        cache_path=str(path))
    assert tuned2 == {"r64-bf16": 221} and fresh[0]["plan"].code == 221
    assert calls == [{64: 221}]


class FakeRowPlan:
    """A plan for tune_plan: FP32 rows, current codes (variant, variant_t)."""

    def __init__(self, current=(32212, 1042)):
        self.m, self.n, self.r, self.nnz = 8, 6, 4, 10
        self.device = torch.device("cpu")
        self.current = current
        self.code = None
        self.set_calls = []

    def info(self):
        return {"variant": self.current[0], "variant_t": self.current[1]}

    def set_variant(self, v, vt):
        self.set_calls.append((v, vt))
        self.code = v


def test_tune_plan_times_the_current_codes_and_keeps_the_fastest(monkeypatch):
    """The plan's current codes are timed with the candidates, so tuning
    never returns a slower variant than the one the plan had; each side
    keeps its own fastest code."""
    plan = FakeRowPlan()
    s_cost = {32212: 1.0, 112: 1.5, 212: 1.2}       # the current S code is fastest
    t_cost = {1042: 2.0, 22412: 1.8, 212: 2.5}      # a candidate beats the current S^T code

    def fake_time(fn, iters):
        table = s_cost if fn.__name__ == "s_side" else t_cost
        return table.get(plan.code, 9.0)

    monkeypatch.setattr(autotune, "_time", fake_time)
    res = autotune.tune_plan(plan, None, None, None, candidates=(112, 212, 22412))
    timed = [v for v, _ in plan.set_calls[:-1]]
    assert set(timed) == {112, 212, 22412, 32212, 1042} and len(timed) == 5
    assert res["variant"] == 32212 and res["variant_t"] == 22412
    assert plan.set_calls[-1] == (32212, 22412)


def test_all_codes_are_known_to_the_library():
    """Every default candidate is a variant code the C ABI accepts (the list
    in fmm_api.cu, mirrored by the parity tests)."""
    import re
    from pathlib import Path
    src = (Path(__file__).resolve().parents[1] / "paper_2203_07673_gb300" / "csrc"
           / "fmm_api.cu").read_text()
    body = src[src.index("kVariantCodes[] = {"):].split("};")[0]
    known = {int(x) for x in re.findall(r"\d+", body.split("{", 1)[1])}
    assert set(autotune.ALL_CODES) <= known
    assert set(autotune.BATCH_CODES) <= known
