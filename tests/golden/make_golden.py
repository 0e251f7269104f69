"""Writes the small regression fixture ``fusedmm_small.txt``.

The expected values come from the FP64 oracle alone (oracle/fmm_oracle.c);
nothing here touches the CUDA library.  The inputs are integers scaled by
1/8 and 1/4, so every value in the file is written exactly.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "fusedmm_small.txt")


def inputs():
    rng = np.random.default_rng(20220315)
    m, n, r = 12, 9, 8
    deg = rng.integers(0, 5, size=m)
    deg[3] = 0
    row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    col_idx = rng.integers(0, n, size=int(row_ptr[-1])).astype(np.int64)
    vals = rng.integers(1, 9, size=col_idx.size) / 4.0
    A = rng.integers(-4, 5, size=(m, r)) / 8.0
    B = rng.integers(-4, 5, size=(n, r)) / 8.0
    return m, n, r, row_ptr, col_idx, vals, A, B


def _row(name, arr):
    flat = np.asarray(arr).reshape(-1)
    return name + " " + " ".join(repr(float(x)) if np.issubdtype(flat.dtype, np.floating)
                                 else str(int(x)) for x in flat)


def write():
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    import oracle
    m, n, r, rp, ci, vals, A, B = inputs()
    out = oracle.fusedmm(rp, ci, vals, A, B, n)
    out_t = oracle.fusedmm_t(rp, ci, vals, A, B, n)
    lines = ["# FusedMMA / FusedMMB regression fixture (Sec. II definitions).",
             "# Written by tests/golden/make_golden.py from the FP64 oracle only.",
             f"dims {m} {n} {r}", _row("row_ptr", rp), _row("col_idx", ci),
             _row("vals", vals), _row("A", A), _row("B", B),
             _row("out", out), _row("out_t", out_t)]
    with open(PATH, "w") as f:
        f.write("\n".join(lines) + "\n")


def read(path=PATH):
    d = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, *rest = line.split()
        d[key] = rest
    m, n, r = (int(x) for x in d["dims"])
    f = lambda k: np.array([float(x) for x in d[k]])
    return dict(m=m, n=n, r=r,
                row_ptr=np.array([int(x) for x in d["row_ptr"]], np.int64),
                col_idx=np.array([int(x) for x in d["col_idx"]], np.int64),
                vals=f("vals"), A=f("A").reshape(m, r), B=f("B").reshape(n, r),
                out=f("out").reshape(m, r), out_t=f("out_t").reshape(n, r))


if __name__ == "__main__":
    write()
