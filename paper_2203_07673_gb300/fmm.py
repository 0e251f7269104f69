"""Thin Python binding of libfmm (the C ABI in include/fmm.h).

Argument marshalling only: every function checks tensor devices, dtypes and
shapes, passes raw device pointers and the current CUDA stream to the C entry
point of the same name, and raises ``FmmError`` on a nonzero status.  All
computation happens in the library's CUDA kernels; there is no CPU path.  If
the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfmm.so")

FMM_OK, FMM_EINVAL, FMM_EUNSUPPORTED, FMM_EOVERFLOW, FMM_ECUDA, FMM_ENOMEM, FMM_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
FMM_F32, FMM_BF16 = 0, 1
FMM_PLAN_NO_TRANSPOSE = 1

# Every function of the C ABI, with its ctypes argument types.
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIGNATURES = {
    "fmm_csr_validate": ([_P, _P, _P], ctypes.c_int),
    "fmm_plan_create": ([_P, _I32, _I32, _P, _P, _P], ctypes.c_int),
    "fmm_plan_destroy": ([_P], ctypes.c_int),
    "fmm_plan_get_info": ([_P, _P], ctypes.c_int),
    "fmm_plan_status": ([_P, _P], ctypes.c_int),
    "fmm_sddmm": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_spmm": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_spmm_t": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_t": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_bwd": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_t_bwd": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_acc": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_sddmm_acc": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_spmm_acc": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_spmm_t_acc": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_t_acc": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_bwd_acc": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_fusedmm_noalloc": ([_P, _I32, _I32, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_plan_set_variant": ([_P, _I32, _I32], ctypes.c_int),
    "fmm_plan_set_values": ([_P, _P, _P], ctypes.c_int),
    "fmm_gat_forward": ([_P, _I32, _P, _P, _P, _P, ctypes.c_float, _P, _P], ctypes.c_int),
    "fmm_gat_project": ([_I32, _I32, _I32, _P, _P, _P, _P], ctypes.c_int),
    "fmm_cg_init": ([_I32, _I32, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_cg_update": ([_I32, _I32, ctypes.c_float, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "fmm_batch_create": ([_P, _I32, _P, _P], ctypes.c_int),
    "fmm_batch_forward": ([_P, _P], ctypes.c_int),
    "fmm_batch_backward": ([_P, _P], ctypes.c_int),
    "fmm_batch_destroy": ([_P], ctypes.c_int),
    "fmm_probe_gather": ([_P, ctypes.c_int64, _I32, _P, ctypes.c_int64, _P, _P], ctypes.c_int),
    "fmm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "fmm_last_error": ([], ctypes.c_char_p),
    "fmm_version": ([], ctypes.c_int32),
}


class FmmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_string(status)}) {detail}".rstrip())


class _Csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("split_nnz", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("r", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("max_row_nnz", ctypes.c_int32), ("max_col_nnz", ctypes.c_int32),
                ("split_rows", ctypes.c_int32), ("split_cols", ctypes.c_int32),
                ("row_chunks", ctypes.c_int32), ("col_chunks", ctypes.c_int32),
                ("split_nnz", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("variant_t", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libfmm (raises if it is not built or cannot be loaded)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libfmm is not built ({LIB_PATH} missing); "
                                   "run __graft_entry__.build() or "
                                   "python -m paper_2203_07673_gb300.build")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(handle, name)
                fn.argtypes = args
                fn.restype = res
            _lib = handle
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().fmm_status_string(int(status)).decode()
    except Exception:  # the library itself is missing
        return "?"


def last_error() -> str:
    return lib().fmm_last_error().decode()


def _check(rc: int, where: str):
    if rc != FMM_OK:
        raise FmmError(rc, where, last_error())


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


_DT = {torch.float32: FMM_F32, torch.bfloat16: FMM_BF16}


def _ptr(t, name, dtype=None, shape=None, device=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the plan on {device}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr() if t.numel() else None


class Plan:
    """A preprocessed sparse pattern (the C ``fmm_plan``).

    ``row_ptr`` (m + 1) and ``col_idx`` (nnz) are int32 CUDA tensors; the plan
    keeps references to them, and they must not be modified while it lives.
    ``dtype`` is the dense operand dtype (torch.float32 or torch.bfloat16).
    """

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, n: int, r: int,
                 dtype=torch.float32, transpose: bool = True, split_nnz: int = 0,
                 variant: int = 0, stream=None):
        if dtype not in _DT:
            raise TypeError(f"unsupported dtype {dtype}")
        self.handle = None
        self.device = row_ptr.device
        _ptr(row_ptr, "row_ptr", torch.int32)
        _ptr(col_idx, "col_idx", torch.int32, device=self.device)
        if row_ptr.dim() != 1 or col_idx.dim() != 1 or row_ptr.numel() < 1:
            raise ValueError("row_ptr and col_idx must be 1-D (row_ptr with m + 1 entries)")
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.m, self.n, self.r = row_ptr.numel() - 1, int(n), int(r)
        self.nnz = col_idx.numel()
        self.dtype = dtype
        csr = _Csr(self.m, self.n, self.nnz, row_ptr.data_ptr(),
                   col_idx.data_ptr() if self.nnz else None)
        opt = _Options(0 if transpose else FMM_PLAN_NO_TRANSPOSE, int(split_nnz), int(variant))
        out = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().fmm_plan_create(ctypes.byref(csr), self.r, _DT[dtype], ctypes.byref(opt),
                                       _stream(stream), ctypes.byref(out))
        _check(rc, "fmm_plan_create")
        self.handle = out.value

    def set_variant(self, variant: int = 0, variant_t: int = 0):
        """fmm_plan_set_variant (0 leaves a side unchanged)."""
        _check(lib().fmm_plan_set_variant(self.handle, int(variant), int(variant_t)),
               "fmm_plan_set_variant")

    def set_values(self, vals, stream=None):
        """fmm_plan_set_values: register values that stay unchanged (None
        forgets them); keeps a reference to the tensor."""
        self._static_vals = vals
        rc = lib().fmm_plan_set_values(self.handle, self._f32(vals, (self.nnz,), "vals"),
                                       _stream(stream))
        _check(rc, "fmm_plan_set_values")

    def status(self, stream=None):
        """fmm_plan_status: synchronise the stream and raise FmmError if a pass
        of this plan gave up a bounded wait (the error word is cleared)."""
        _check(lib().fmm_plan_status(self.handle, _stream(stream)), "fmm_plan_status")

    def info(self) -> dict:
        inf = _Info()
        _check(lib().fmm_plan_get_info(self.handle, ctypes.byref(inf)), "fmm_plan_get_info")
        return {name: getattr(inf, name) for name, _ in _Info._fields_}

    def close(self):
        if self.handle is not None:
            lib().fmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shape helpers
    def _dense(self, t, rows, name):
        return _ptr(t, name, self.dtype, (rows, self.r), self.device)

    def _f32(self, t, shape, name):
        return _ptr(t, name, torch.float32, shape, self.device)


def validate(row_ptr: torch.Tensor, col_idx: torch.Tensor, n: int, stream=None) -> int:
    """fmm_csr_validate: -1 if valid, else the first bad index (see fmm.h)."""
    csr = _Csr(row_ptr.numel() - 1, int(n), col_idx.numel(), row_ptr.data_ptr(),
               col_idx.data_ptr() if col_idx.numel() else None)
    bad = ctypes.c_int64(-1)
    rc = lib().fmm_csr_validate(ctypes.byref(csr), _stream(stream), ctypes.byref(bad))
    if rc not in (FMM_OK, FMM_EINVAL):
        _check(rc, "fmm_csr_validate")
    return int(bad.value)


def _out(out, shape, plan):
    if out is None:
        return torch.empty(shape, dtype=torch.float32, device=plan.device)
    return out


def sddmm(plan: Plan, vals, A, B, out=None, stream=None):
    out = _out(out, (plan.nnz,), plan)
    rc = lib().fmm_sddmm(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                         plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                         plan._f32(out, (plan.nnz,), "out"), _stream(stream))
    _check(rc, "fmm_sddmm")
    return out


def spmm(plan: Plan, v, B, out=None, stream=None):
    out = _out(out, (plan.m, plan.r), plan)
    rc = lib().fmm_spmm(plan.handle, plan._f32(v, (plan.nnz,), "v"),
                        plan._dense(B, plan.n, "B"), plan._f32(out, (plan.m, plan.r), "out"),
                        _stream(stream))
    _check(rc, "fmm_spmm")
    return out


def spmm_t(plan: Plan, v, A, out=None, stream=None):
    out = _out(out, (plan.n, plan.r), plan)
    rc = lib().fmm_spmm_t(plan.handle, plan._f32(v, (plan.nnz,), "v"),
                          plan._dense(A, plan.m, "A"), plan._f32(out, (plan.n, plan.r), "out"),
                          _stream(stream))
    _check(rc, "fmm_spmm_t")
    return out


def fusedmm(plan: Plan, vals, A, B, out=None, stream=None):
    out = _out(out, (plan.m, plan.r), plan)
    rc = lib().fmm_fusedmm(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                           plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                           plan._f32(out, (plan.m, plan.r), "out"), _stream(stream))
    _check(rc, "fmm_fusedmm")
    return out


def fusedmm_t(plan: Plan, vals, A, B, out=None, stream=None):
    out = _out(out, (plan.n, plan.r), plan)
    rc = lib().fmm_fusedmm_t(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                             plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                             plan._f32(out, (plan.n, plan.r), "out"), _stream(stream))
    _check(rc, "fmm_fusedmm_t")
    return out


def fusedmm_bwd(plan: Plan, vals, A, B, G, need=(True, True, True), stream=None, out=None):
    """Returns (dA, dB, ds) (float32; None where need is False).  `out`, if
    given, is (dA, dB, ds) to write into (None entries are skipped)."""
    if out is not None:
        dA, dB, ds = out
    else:
        dA = (torch.empty((plan.m, plan.r), dtype=torch.float32, device=plan.device)
              if need[0] else None)
        dB = (torch.empty((plan.n, plan.r), dtype=torch.float32, device=plan.device)
              if need[1] else None)
        ds = torch.empty((plan.nnz,), dtype=torch.float32, device=plan.device) if need[2] else None
    rc = lib().fmm_fusedmm_bwd(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                               plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                               plan._f32(G, (plan.m, plan.r), "G"),
                               plan._f32(dA, (plan.m, plan.r), "dA"),
                               plan._f32(dB, (plan.n, plan.r), "dB"),
                               plan._f32(ds, (plan.nnz,), "ds"), _stream(stream))
    _check(rc, "fmm_fusedmm_bwd")
    return dA, dB, ds


def sddmm_acc(plan: Plan, vals, A, B, v, stream=None):
    """fmm_sddmm_acc: v += SDDMM (v float32, nnz, valid values)."""
    rc = lib().fmm_sddmm_acc(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                             plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                             plan._f32(v, (plan.nnz,), "v"), _stream(stream))
    _check(rc, "fmm_sddmm_acc")
    return v


def spmm_acc(plan: Plan, v, B, out, stream=None):
    """fmm_spmm_acc: out += SpMMA(v, B) (out float32, m x r)."""
    rc = lib().fmm_spmm_acc(plan.handle, plan._f32(v, (plan.nnz,), "v"),
                            plan._dense(B, plan.n, "B"), plan._f32(out, (plan.m, plan.r), "out"),
                            _stream(stream))
    _check(rc, "fmm_spmm_acc")
    return out


def spmm_t_acc(plan: Plan, v, A, out, stream=None):
    """fmm_spmm_t_acc: out += SpMMB(v, A) (out float32, n x r)."""
    rc = lib().fmm_spmm_t_acc(plan.handle, plan._f32(v, (plan.nnz,), "v"),
                              plan._dense(A, plan.m, "A"), plan._f32(out, (plan.n, plan.r), "out"),
                              _stream(stream))
    _check(rc, "fmm_spmm_t_acc")
    return out


def fusedmm_acc(plan: Plan, vals, A, B, out, stream=None):
    """fmm_fusedmm_acc: out += FusedMMA (out float32, m x r, valid values)."""
    rc = lib().fmm_fusedmm_acc(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                               plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                               plan._f32(out, (plan.m, plan.r), "out"), _stream(stream))
    _check(rc, "fmm_fusedmm_acc")
    return out


def fusedmm_t_acc(plan: Plan, vals, A, B, out, stream=None):
    """fmm_fusedmm_t_acc: out += FusedMMB (out float32, n x r, valid values)."""
    rc = lib().fmm_fusedmm_t_acc(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                                 plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                                 plan._f32(out, (plan.n, plan.r), "out"), _stream(stream))
    _check(rc, "fmm_fusedmm_t_acc")
    return out


def fusedmm_bwd_acc(plan: Plan, vals, A, B, G, dA=None, dB=None, ds=None, stream=None):
    """fmm_fusedmm_bwd_acc: dA += and dB += the adjoint of FusedMMA, ds =
    (each may be None to skip it)."""
    rc = lib().fmm_fusedmm_bwd_acc(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                                   plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                                   plan._f32(G, (plan.m, plan.r), "G"),
                                   plan._f32(dA, (plan.m, plan.r), "dA"),
                                   plan._f32(dB, (plan.n, plan.r), "dB"),
                                   plan._f32(ds, (plan.nnz,), "ds"), _stream(stream))
    _check(rc, "fmm_fusedmm_bwd_acc")
    return dA, dB, ds


def fusedmm_t_bwd(plan: Plan, vals, A, B, Gn, need=(True, True, True), stream=None):
    """Returns (dA, dB, ds) for L = <Gn, FusedMMB>."""
    dA = torch.empty((plan.m, plan.r), dtype=torch.float32, device=plan.device) if need[0] else None
    dB = torch.empty((plan.n, plan.r), dtype=torch.float32, device=plan.device) if need[1] else None
    ds = torch.empty((plan.nnz,), dtype=torch.float32, device=plan.device) if need[2] else None
    rc = lib().fmm_fusedmm_t_bwd(plan.handle, plan._f32(vals, (plan.nnz,), "vals"),
                                 plan._dense(A, plan.m, "A"), plan._dense(B, plan.n, "B"),
                                 plan._f32(Gn, (plan.n, plan.r), "Gn"),
                                 plan._f32(dA, (plan.m, plan.r), "dA"),
                                 plan._f32(dB, (plan.n, plan.r), "dB"),
                                 plan._f32(ds, (plan.nnz,), "ds"), _stream(stream))
    _check(rc, "fmm_fusedmm_t_bwd")
    return dA, dB, ds


def fusedmm_noalloc(row_ptr, col_idx, n: int, vals, A, B, out=None, stream=None):
    """fmm_fusedmm_noalloc: FusedMMA from the CSR directly, with no plan and
    no device allocation inside the library (``out`` is allocated here by
    torch if not given).  Every tensor must be on A's device, which is made
    current for the call.  Calls that overlap on the GPU must not be issued:
    they share one fixed scratch array."""
    if not isinstance(A, torch.Tensor) or A.dim() != 2:
        raise ValueError("A must be a 2-D tensor (m x r)")
    dt = _DT.get(A.dtype)
    if dt is None:
        raise TypeError(f"unsupported dtype {A.dtype}")
    dev = A.device
    m, r = A.shape
    if not isinstance(row_ptr, torch.Tensor) or row_ptr.dim() != 1 or row_ptr.numel() != m + 1:
        raise ValueError(f"row_ptr must be 1-D with m + 1 = {m + 1} entries")
    if not isinstance(col_idx, torch.Tensor) or col_idx.dim() != 1:
        raise ValueError("col_idx must be 1-D")
    nnz = col_idx.numel()
    if out is None:
        out = torch.empty((m, r), dtype=torch.float32, device=dev)
    csr = _Csr(m, int(n), nnz, _ptr(row_ptr, "row_ptr", torch.int32, device=dev),
               _ptr(col_idx, "col_idx", torch.int32, device=dev))
    args = (_ptr(vals, "vals", torch.float32, (nnz,), device=dev),
            _ptr(A, "A", device=dev), _ptr(B, "B", A.dtype, (int(n), r), device=dev),
            _ptr(out, "out", torch.float32, (m, r), device=dev))
    with torch.cuda.device(dev):
        rc = lib().fmm_fusedmm_noalloc(ctypes.byref(csr), int(r), dt, *args, _stream(stream))
    _check(rc, "fmm_fusedmm_noalloc")
    return out


def probe_gather(table, idx, sink=None, stream=None):
    """fmm_probe_gather: fetch table[idx[k]] for every k and nothing else (a
    measurement aid: the gather ceiling of a pass walking idx).  table is a
    2-D contiguous CUDA tensor whose rows are 64, 128, 256 or 512 bytes;
    idx int32 on the same device."""
    if not isinstance(table, torch.Tensor) or table.dim() != 2:
        raise ValueError("table must be a 2-D tensor")
    dev = table.device
    row_bytes = table.shape[1] * table.element_size()
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int32, device=dev)
    args = (_ptr(table, "table", device=dev), table.shape[0], row_bytes,
            _ptr(idx, "idx", torch.int32, device=dev), idx.numel(),
            _ptr(sink, "sink", device=dev))
    with torch.cuda.device(dev):
        rc = lib().fmm_probe_gather(*args, _stream(stream))
    _check(rc, "fmm_probe_gather")


class _BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("out", ctypes.c_void_p), ("G", ctypes.c_void_p),
                ("dA", ctypes.c_void_p), ("dB", ctypes.c_void_p), ("ds", ctypes.c_void_p)]


class Batch:
    """fmm_batch: FusedMMA (and its adjoint) of many plans in one persistent
    launch per phase.  ``items`` is a list of dicts with keys plan, vals, A,
    B, out and optionally G, dA, dB, ds (tensors on the plans' device).  The
    batch keeps references to every tensor; their storage must not move."""

    def __init__(self, items, stream=None):
        self.handle = None
        self._keep = items
        arr = (_BatchItem * len(items))()
        for k, it in enumerate(items):
            p = it["plan"]
            arr[k] = _BatchItem(
                p.handle, p._f32(it.get("vals"), (p.nnz,), "vals"), p._dense(it["A"], p.m, "A"),
                p._dense(it["B"], p.n, "B"), p._f32(it["out"], (p.m, p.r), "out"),
                p._f32(it.get("G"), (p.m, p.r), "G"), p._f32(it.get("dA"), (p.m, p.r), "dA"),
                p._f32(it.get("dB"), (p.n, p.r), "dB"), p._f32(it.get("ds"), (p.nnz,), "ds"))
        out = ctypes.c_void_p()
        rc = lib().fmm_batch_create(arr, len(items), _stream(stream), ctypes.byref(out))
        _check(rc, "fmm_batch_create")
        self.handle = out.value

    def forward(self, stream=None):
        _check(lib().fmm_batch_forward(self.handle, _stream(stream)), "fmm_batch_forward")

    def backward(self, stream=None):
        _check(lib().fmm_batch_backward(self.handle, _stream(stream)), "fmm_batch_backward")

    def close(self):
        if self.handle is not None:
            lib().fmm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rows_f32(t, rows, r, name):
    return _ptr(t, name, torch.float32, (rows, r))


def cg_init(lam, b, mx, x, res, p, rs, stream=None):
    """fmm_cg_init on float32 row blocks (rows x r)."""
    rows, r = x.shape
    rc = lib().fmm_cg_init(rows, r, float(lam), _rows_f32(b, rows, r, "b"),
                           _rows_f32(mx, rows, r, "mx"), _rows_f32(x, rows, r, "x"),
                           _rows_f32(res, rows, r, "res"), _rows_f32(p, rows, r, "p"),
                           _ptr(rs, "rs", torch.float32, (rows,)), _stream(stream))
    _check(rc, "fmm_cg_init")


def cg_update(lam, x, res, p, q, rs, stream=None):
    """fmm_cg_update on float32 row blocks (rows x r)."""
    rows, r = x.shape
    rc = lib().fmm_cg_update(rows, r, float(lam), _rows_f32(x, rows, r, "x"),
                             _rows_f32(res, rows, r, "res"), _rows_f32(p, rows, r, "p"),
                             _rows_f32(q, rows, r, "q"), _ptr(rs, "rs", torch.float32, (rows,)),
                             _stream(stream))
    _check(rc, "fmm_cg_update")


def gat_project(X, w, heads, out=None, stream=None):
    """fmm_gat_project: per-head projections X[:, head] . w[head] (float32)."""
    rows, r = X.shape
    if out is None:
        out = torch.empty(rows, heads, dtype=torch.float32, device=X.device)
    rc = lib().fmm_gat_project(rows, heads, r // heads, _ptr(X, "X", torch.float32, (rows, r)),
                               _ptr(w, "w", torch.float32, (r,)),
                               _ptr(out, "out", torch.float32, (rows, heads)), _stream(stream))
    _check(rc, "fmm_gat_project")
    return out


def gat_forward(plan: Plan, heads, vals, f, g, H, slope=0.2, out=None, stream=None):
    """fmm_gat_forward: attention scores, row softmax and aggregation."""
    out = _out(out, (plan.m, plan.r), plan)
    rc = lib().fmm_gat_forward(plan.handle, int(heads), plan._f32(vals, (plan.nnz,), "vals"),
                               plan._f32(f, (plan.m, heads), "f"),
                               plan._f32(g, (plan.n, heads), "g"), plan._dense(H, plan.n, "H"),
                               float(slope), plan._f32(out, (plan.m, plan.r), "out"),
                               _stream(stream))
    _check(rc, "fmm_gat_forward")
    return out
