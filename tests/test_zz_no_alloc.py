"""fmm_fusedmm_noalloc: FusedMMA for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they need FusedMMA (code inside a
pool or arena that owns all device memory, or a runtime that forbids
allocation on its hot path); they cannot create a plan, because plan creation
allocates.  This entry point takes the CSR directly and keeps its only scratch
(chunk list and partial rows of long rows) in a fixed file-scope device array.

The test calls it through the C ABI, twice in a row on the same inputs and
once more on a different pattern, and checks each result against the plan
path (fmm_fusedmm) with the tolerance the parity tests use.  The patterns
include rows longer than the chunk size, so the scratch array is exercised,
and the second call checks that state left by the first is cleared.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, relF, upload
from paper_2203_07673_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pattern(seed):
    rng = np.random.default_rng(seed)
    return wl.random_csr(700, 520, rng, mean_deg=9, empty_frac=0.15, dup_frac=0.1,
                         unsorted=True, hubs=((4, 3000), (311, 1400), (699, 600)))


def _noalloc(fmm, S, rp, ci, r, dtype_code, vt, At, Bt, out):
    csr = fmm._Csr(S.m, S.n, S.nnz, rp.data_ptr(), ci.data_ptr())
    rc = fmm.lib().fmm_fusedmm_noalloc(ctypes.byref(csr), r, dtype_code,
                                       vt.data_ptr() if vt is not None else None,
                                       At.data_ptr(), Bt.data_ptr(), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == fmm.FMM_OK, fmm.last_error()
    return out


def _close_to_plan_path(name, got, ref, mag, r, deg):
    # both results are float32 sums of the same terms in different orders:
    # each lies within the rounding bound of the exact value, so their
    # difference lies within twice that bound
    got = got.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    bound = 2 * 2.0 * (r + deg + 4) * U32 * mag + 1e-30
    assert np.all(np.abs(got - ref) <= bound), name
    assert relF(got, ref) <= 1e-5, name


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("r", [64, 128, 24])
def test_noalloc_matches_plan_path_on_two_calls(r, dtype):
    from paper_2203_07673_gb300 import fmm
    code = fmm.FMM_F32 if dtype == torch.float32 else fmm.FMM_BF16
    results = []
    for seed in (1, 1, 2):          # two calls in a row on one pattern, then another pattern
        S = _pattern(seed)
        rng = np.random.default_rng(seed + 10)
        vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
        A = (rng.standard_normal((S.m, r)) / np.sqrt(r)).astype(np.float32)
        B = (rng.standard_normal((S.n, r)) / np.sqrt(r)).astype(np.float32)
        rp, ci, vt, At, Bt = upload(S, vals, A, B, dtype)
        plan = fmm.Plan(rp, ci, S.n, r, dtype)
        ref = fmm.fusedmm(plan, vt, At, Bt)
        out = torch.full((S.m, r), float("nan"), device="cuda")
        _noalloc(fmm, S, rp, ci, r, code, vt, At, Bt, out)
        torch.cuda.synchronize()
        mag = oracle.fusedmm(S.row_ptr, S.col_idx, vals, np.abs(At.double().cpu().numpy()),
                             np.abs(Bt.double().cpu().numpy()), S.n)
        deg = int(S.degrees().max())
        _close_to_plan_path(f"noalloc seed {seed}", out, ref, mag, r, deg)
        results.append(out.clone())
        plan.close()
    # the same inputs give the same bits on the repeated call
    assert torch.equal(results[0], results[1])


def test_noalloc_rejects_oversized_r():
    from paper_2203_07673_gb300 import fmm
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    csr = fmm._Csr(1, 1, 0, rp.data_ptr(), None)
    buf = torch.zeros(16, device="cuda")
    rc = fmm.lib().fmm_fusedmm_noalloc(ctypes.byref(csr), (1 << 16) + 1, fmm.FMM_F32, None,
                                       buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
    assert rc == fmm.FMM_EOVERFLOW
    assert b"65536" in fmm.lib().fmm_last_error()
