"""CPU checks of bench.py's byte models and the traffic lookup."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2203_07673_gb300 import workloads as wl  # noqa: E402


class _S:
    def __init__(self, m, n, nnz):
        self.m, self.n, self.nnz = m, n, nnz


def test_gather_model_counts_every_stream():
    m, nnz, r, e = 10, 37, 16, 4
    # row_ptr, col_idx, values, local rows, one gathered row per nonzero, output
    want = 4 * (m + 1) + 4 * nnz + 4 * nnz + m * r * e + nnz * r * e + 4 * m * r
    assert bench.gather_model_bytes(m, nnz, r, e) == want
    assert bench.gather_model_bytes(m, nnz, r, e, vals=False) == want - 4 * nnz


def test_compulsory_model_reads_each_dense_row_once():
    m, n, nnz, r, e = 10, 7, 37, 16, 2
    g = bench.gather_model_bytes(m, nnz, r, e)
    c = bench.compulsory_model_bytes(m, n, nnz, r, e)
    assert g - c == (nnz - n) * r * e


def test_step_calls_of_the_forward_step():
    S, r, e = _S(10, 7, 37), 16, 4
    calls = dict(bench.step_calls(2, S, r, e, True))
    assert calls["fmm_fusedmm"] == bench.gather_model_bytes(10, 37, r, e)
    # the pass over S^T gathers rows of A per nonzero and permutes the values
    assert calls["fmm_fusedmm_t"] == bench.gather_model_bytes(7, 37, r, e) + 12 * 37
    comp = dict(bench.step_calls(2, S, r, e, True, bench.compulsory_model_bytes))
    assert comp["fmm_fusedmm_t"] == bench.compulsory_model_bytes(7, 10, 37, r, e) + 12 * 37


def test_step_calls_of_the_backward_step():
    S, r, e = _S(10, 7, 37), 16, 2
    calls = dict(bench.step_calls(3, S, r, e, True))
    p1 = bench.gather_model_bytes(10, 37, r, e) + 4 * 10 * r + 4 * 37
    p2 = bench.gather_model_bytes(7, 37, r, e) + 4 * 37 * r + 12 * 37
    assert calls["fmm_fusedmm_bwd"] == p1 + p2


def test_traffic_lookup_needs_matching_sources(tmp_path, monkeypatch):
    name = wl.WORKLOADS[2]
    good = tmp_path / "good.txt"
    good.write_text(f"# header\n{name} | fmm_fusedmm | f32 | 123 | {bench.kernel_source_sha()} | k\n")
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(good))
    assert bench.read_traffic(name, "fmm_fusedmm", "f32") == (123.0, "k")
    assert bench.read_traffic(name, "fmm_fusedmm_t", "f32")[0] is None
    stale = tmp_path / "stale.txt"
    stale.write_text(f"{name} | fmm_fusedmm | f32 | 123 | {'0' * 40} | k\n")
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(stale))
    v, note = bench.read_traffic(name, "fmm_fusedmm", "f32")
    assert v is None and "predates" in note


@pytest.mark.parametrize("k", [2, 3, 4])
def test_committed_traffic_file_parses(k):
    """profiles/roofline_traffic.txt holds a line for every bench call."""
    calls = {2: "fmm_fusedmm_t", 3: "fmm_fusedmm_bwd", 4: "fmm_fusedmm_t"}
    dtype = "bf16" if k == 3 else "f32"
    found = False
    with open(bench.PROFILE_TRAFFIC) as fh:
        for line in fh:
            f = [x.strip() for x in line.split("|")]
            if len(f) >= 6 and f[0] == wl.WORKLOADS[k] and f[1] == calls[k] and f[2] == dtype:
                found = float(f[3]) > 0 and len(f[4]) == 40
    assert found
