"""fmm_fusedmm_noalloc: FusedMMA for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they need FusedMMA (code inside a
pool or arena that owns all device memory, or a runtime that forbids
allocation on its hot path); they cannot create a plan, because plan creation
allocates.  This entry point takes the CSR directly and keeps its only scratch
(chunk list and partial rows of long rows) in a fixed file-scope device array.

The tests call it through the C ABI and through the Python wrapper, twice in a
row on the same inputs and once more on a different pattern, and check every
element of each result against the FP64 oracle with the rounding bound of
the parity tests (and against the plan path, fmm_fusedmm, with twice that
bound).  The patterns include rows longer than the chunk size, so the scratch
array is exercised, and the repeated call checks that state left by the
first is cleared.  One pattern is large enough (11.8M nonzeros at r = 256)
that the chunk size grows past its 512 minimum to keep every chunk inside
the fixed array.  This file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity_utils import U32, assert_close, host64, relF, rows_problem, upload
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
def test_noalloc_matches_oracle_on_two_calls(r, dtype):
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
        out = torch.full((S.m, r), float("nan"), device="cuda")
        _noalloc(fmm, S, rp, ci, r, code, vt, At, Bt, out)
        torch.cuda.synchronize()
        # the oracle on exactly the values the GPU received (bf16 widened)
        A64, B64 = host64(At), host64(Bt)
        exp = oracle.fusedmm(S.row_ptr, S.col_idx, vals, A64, B64, S.n)
        mag = oracle.fusedmm(S.row_ptr, S.col_idx, vals, np.abs(A64), np.abs(B64), S.n)
        deg = int(S.degrees().max())
        assert_close(f"noalloc seed {seed}", out, exp, mag, r, deg)
        # and the plan path on the same inputs
        plan = fmm.Plan(rp, ci, S.n, r, dtype)
        ref = fmm.fusedmm(plan, vt, At, Bt)
        _close_to_plan_path(f"noalloc vs plan seed {seed}", out, ref, mag, r, deg)
        results.append(out.clone())
        plan.close()
    # the same inputs give the same bits on the repeated call
    assert torch.equal(results[0], results[1])


def test_noalloc_wrapper_chunk_size_above_minimum():
    """Through fmm.fusedmm_noalloc: 2^17 rows of about 90 nonzeros plus hub
    rows of 3000 and 5000 at r = 256, so the chunk size is
    ch = ceil(2 nnz / (8 Mi / r)) > 512; sampled rows (the hub rows among
    them) against the oracle, and a repeated call bit for bit."""
    from paper_2203_07673_gb300 import fmm
    r, m, n = 256, 1 << 17, 1 << 16
    rng = np.random.default_rng(77)
    S = wl.random_csr(m, n, rng, mean_deg=90, empty_frac=0.02,
                      hubs=((5, 3000), (70000, 5000), (m - 1, 3000)))
    cap = min(1 << 16, (1 << 23) // r)
    ch = max(512, -(-2 * S.nnz // cap))
    assert ch > 512 and S.degrees().max() > ch
    vals = rng.uniform(0, 1, S.nnz).astype(np.float32)
    A = wl.normal(m, r, 1.0 / r, rng)
    B = wl.normal(n, r, 1.0 / r, rng)
    rp, ci, vt, At, Bt = upload(S, vals, A, B)
    out1 = fmm.fusedmm_noalloc(rp, ci, n, vt, At, Bt)
    out2 = torch.full_like(out1, float("nan"))
    fmm.fusedmm_noalloc(rp, ci, n, vt, At, Bt, out=out2)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)
    rows = np.unique(np.concatenate([[5, 70000, m - 1],
                                     np.random.default_rng(3).choice(m, 64, replace=False)]))
    sub_rp, sub_ci, sub_v, cols, _ = rows_problem(S, rows, vals)
    exp = oracle.fusedmm(sub_rp, sub_ci, sub_v, A[rows], B[cols], len(cols))
    mag = oracle.fusedmm(sub_rp, sub_ci, sub_v, np.abs(A[rows]), np.abs(B[cols]), len(cols))
    deg = int(S.degrees()[rows].max())
    assert_close("noalloc r=256 sampled rows", out1[torch.from_numpy(rows).cuda()], exp, mag, r,
                 deg)


def test_noalloc_wrapper_checks_its_arguments():
    from paper_2203_07673_gb300 import fmm
    S = _pattern(3)
    r = 32
    rng = np.random.default_rng(4)
    A = rng.standard_normal((S.m, r)).astype(np.float32)
    B = rng.standard_normal((S.n, r)).astype(np.float32)
    rp, ci, vt, At, Bt = upload(S, None, A, B)
    with pytest.raises(ValueError):
        fmm.fusedmm_noalloc(rp[:-1], ci, S.n, None, At, Bt)        # row_ptr too short
    with pytest.raises(ValueError):
        fmm.fusedmm_noalloc(rp, ci, S.n, None, At, Bt[:-1])        # B has n - 1 rows
    with pytest.raises(ValueError):
        fmm.fusedmm_noalloc(rp, ci, S.n, torch.ones(S.nnz - 1, device="cuda"), At, Bt)
    with pytest.raises(TypeError):
        fmm.fusedmm_noalloc(rp, ci, S.n, None, At, Bt.to(torch.bfloat16))


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
