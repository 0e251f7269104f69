"""FP64 CPU oracle for FusedMM (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
leg of ``bench.py`` may import this package.  The product library never does:
it shares no code with the oracle, and the oracle shares none with it.

The arithmetic lives in ``fmm_oracle.c`` (plain C loops in FP64, each routine
citing the passage of the paper it writes out).  This module only compiles it
with gcc, loads it with ctypes and marshals numpy arrays: indices are widened
to int64 and every floating-point input to float64 before the call.

Functions (all return float64 numpy arrays):
  sddmm(rowptr, colidx, vals, A, B, n)        -> v[nnz]        Sec. II, Eq. (1)
  spmm(rowptr, colidx, v, B, n)               -> out[m, r]     Sec. II (SpMMA)
  spmm_t(rowptr, colidx, v, A, n)             -> out[n, r]     Sec. II (SpMMB)
  fusedmm(rowptr, colidx, vals, A, B, n)      -> out[m, r]     Sec. II / IV-B
  fusedmm_t(rowptr, colidx, vals, A, B, n)    -> out[n, r]     Sec. II (FusedMMB)
  fusedmm_grad(rowptr, colidx, vals, A, B, G, n)     -> (dA, dB, ds)
  fusedmm_t_grad(rowptr, colidx, vals, A, B, Gn, n)  -> (dA, dB, ds)
  als_cg(rowptr, colidx, c, A, B, lam, iters, side)  -> updated A (side 0) or B (side 1)
  als_cg_state(rowptr, colidx, c, A, B, lam, iters, side, state=None)
                                              -> (X, res, p, rs): the same CG with its state
  gat(rowptr, colidx, vals, f, g, H, heads, slope)   -> out[m, heads * rh]  (GAT forward)
``vals=None`` means every value of S is 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile fmm_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_oracle()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, ptr = ctypes.c_int64, ctypes.c_void_p
        sig = {
            "oracle_sddmm": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr, ptr],
            "oracle_spmm": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr],
            "oracle_spmm_t": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr],
            "oracle_fusedmm": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr, ptr],
            "oracle_fusedmm_t": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr, ptr],
            "oracle_fusedmm_grad": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr,
                                    ptr, ptr, ptr, ptr],
            "oracle_fusedmm_t_grad": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr,
                                      ptr, ptr, ptr, ptr],
            "oracle_als_cg": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr, ctypes.c_double,
                              i64, ctypes.c_int],
            "oracle_als_cg_state": [i64, i64, i64, ptr, ptr, ptr, ptr, ptr,
                                    ctypes.c_double, i64, ctypes.c_int, ctypes.c_int,
                                    ptr, ptr, ptr],
            "oracle_gat": [i64, i64, i64, i64, ptr, ptr, ptr, ptr, ptr, ptr, ctypes.c_double,
                           ptr],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.oracle_threads.argtypes = [ctypes.c_int]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def threads(n: int = 0) -> int:
    """Threads of the oracle's parallel row loops: sets the count when
    n > 0; returns the count in effect."""
    return int(_load().oracle_threads(int(n)))


def _i64(x):
    return np.ascontiguousarray(np.asarray(x), dtype=np.int64)


def _f64(x):
    if x is None:
        return None
    if hasattr(x, "detach"):  # a torch tensor (e.g. bf16): widen exactly
        x = x.detach().cpu().double().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data


def _prep(rowptr, colidx, r_from):
    rowptr, colidx = _i64(rowptr), _i64(colidx)
    m = rowptr.shape[0] - 1
    return rowptr, colidx, m


def _dims(X, rows):
    X = _f64(X)
    if X.ndim != 2 or X.shape[0] != rows:
        raise ValueError(f"expected a {rows} x r matrix, got {X.shape}")
    return X


def _run(fn, *args):
    rc = fn(*args)
    if rc != 0:
        raise ValueError("oracle: malformed CSR (index out of range)")


def sddmm(rowptr, colidx, vals, A, B, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, B = _dims(A, m), _dims(B, n)
    vals = _f64(vals)
    r = A.shape[1]
    v = np.zeros(colidx.shape[0], np.float64)
    _run(_load().oracle_sddmm, m, n, r, _p(rowptr), _p(colidx), _p(vals),
         _p(A), _p(B), _p(v))
    return v


def spmm(rowptr, colidx, v, B, n):
    rowptr, colidx, m = _prep(rowptr, colidx, B)
    B, v = _dims(B, n), _f64(v)
    r = B.shape[1]
    out = np.zeros((m, r), np.float64)
    _run(_load().oracle_spmm, m, n, r, _p(rowptr), _p(colidx), _p(v), _p(B),
         _p(out))
    return out


def spmm_t(rowptr, colidx, v, A, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, v = _dims(A, m), _f64(v)
    r = A.shape[1]
    out = np.zeros((n, r), np.float64)
    _run(_load().oracle_spmm_t, m, n, r, _p(rowptr), _p(colidx), _p(v), _p(A),
         _p(out))
    return out


def fusedmm(rowptr, colidx, vals, A, B, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, B, vals = _dims(A, m), _dims(B, n), _f64(vals)
    r = A.shape[1]
    out = np.zeros((m, r), np.float64)
    _run(_load().oracle_fusedmm, m, n, r, _p(rowptr), _p(colidx), _p(vals),
         _p(A), _p(B), _p(out))
    return out


def fusedmm_t(rowptr, colidx, vals, A, B, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, B, vals = _dims(A, m), _dims(B, n), _f64(vals)
    r = A.shape[1]
    out = np.zeros((n, r), np.float64)
    _run(_load().oracle_fusedmm_t, m, n, r, _p(rowptr), _p(colidx), _p(vals),
         _p(A), _p(B), _p(out))
    return out


def fusedmm_grad(rowptr, colidx, vals, A, B, G, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, B, G, vals = _dims(A, m), _dims(B, n), _dims(G, m), _f64(vals)
    r = A.shape[1]
    dA = np.zeros((m, r)); dB = np.zeros((n, r))
    ds = np.zeros(colidx.shape[0])
    _run(_load().oracle_fusedmm_grad, m, n, r, _p(rowptr), _p(colidx),
         _p(vals), _p(A), _p(B), _p(G), _p(dA), _p(dB), _p(ds))
    return dA, dB, ds


def fusedmm_t_grad(rowptr, colidx, vals, A, B, Gn, n):
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A, B, Gn, vals = _dims(A, m), _dims(B, n), _dims(Gn, n), _f64(vals)
    r = A.shape[1]
    dA = np.zeros((m, r)); dB = np.zeros((n, r))
    ds = np.zeros(colidx.shape[0])
    _run(_load().oracle_fusedmm_t_grad, m, n, r, _p(rowptr), _p(colidx),
         _p(vals), _p(A), _p(B), _p(Gn), _p(dA), _p(dB), _p(ds))
    return dA, dB, ds


def als_cg(rowptr, colidx, c, A, B, lam, iters, side):
    """`iters` CG iterations per row of the ALS normal equations (Sec. VI-E),
    started from the current rows; returns the updated copy of A (side 0) or
    B (side 1)."""
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A = _dims(A, m).copy()
    B = _f64(B).copy()
    n = B.shape[0]
    c = _f64(c)
    r = A.shape[1]
    _run(_load().oracle_als_cg, m, n, r, _p(rowptr), _p(colidx), _p(c), _p(A), _p(B),
         float(lam), int(iters), int(side))
    return A if side == 0 else B


def als_cg_state(rowptr, colidx, c, A, B, lam, iters, side, state=None):
    """The CG of als_cg with its state exposed (Sec. VI-E).  With state=None
    it starts from the current rows of the side (r = b - M x, p = r,
    rs = <r, r>) and runs `iters` iterations; with state=(res, p, rs) it
    continues from that state (c is then not read).  Returns
    (X, res, p, rs): the updated side and the state after the last
    iteration, all float64 copies."""
    rowptr, colidx, m = _prep(rowptr, colidx, A)
    A = _dims(A, m).copy()
    B = _f64(B).copy()
    n = B.shape[0]
    r = A.shape[1]
    rows = m if side == 0 else n
    if state is None:
        res, p, rs = np.zeros((rows, r)), np.zeros((rows, r)), np.zeros(rows)
        init = 1
        c = _f64(c)
    else:
        res = _f64(state[0]).reshape(rows, r).copy()
        p = _f64(state[1]).reshape(rows, r).copy()
        rs = _f64(state[2]).reshape(rows).copy()
        init = 0
        c = None
    _run(_load().oracle_als_cg_state, m, n, r, _p(rowptr), _p(colidx), _p(c), _p(A), _p(B),
         float(lam), int(iters), int(side), init, _p(res), _p(p), _p(rs))
    return (A if side == 0 else B), res, p, rs


def gat(rowptr, colidx, vals, f, g, H, heads, slope):
    """Multi-head graph-attention forward (Sec. VI-E): f (m x heads), g
    (n x heads), H (n x heads*rh); returns out (m x heads*rh)."""
    rowptr, colidx = _i64(rowptr), _i64(colidx)
    m = rowptr.shape[0] - 1
    f = _f64(f).reshape(m, heads)
    H = _f64(H)
    n = H.shape[0]
    g = _f64(g).reshape(n, heads)
    vals = _f64(vals)          # kept alive across the call
    r = H.shape[1]
    rh = r // heads
    out = np.zeros((m, r))
    _run(_load().oracle_gat, m, n, heads, rh, _p(rowptr), _p(colidx), _p(vals),
         _p(f), _p(g), _p(H), float(slope), _p(out))
    return out
