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
