"""Floating-point operation counts of the oracle (test infrastructure only).

opcount.cpp compiles rhd_oracle.c unchanged with every double replaced by a counting value type
(same arithmetic, same order, same branches).  `bulk_ops_per_cell` runs one subcycle of a workload
at several grid sizes and fits the counts as a cubic in the grid size N: the oracle sweeps one block
of N^3 cells with a two-cell halo, so every loop count is a polynomial of degree 3 in N, and the
N^3 coefficient is the work per cell-update of an unbounded grid (halo work excluded).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "opcount.cpp")
LIB = os.path.join(HERE, "librhd_opcount.so")
CLASSES = ("add", "mul", "div", "sqrt", "cmp", "abs")

_lib = None


def build(force=False):
    deps = [SRC, os.path.join(HERE, "rhd_oracle.c"), os.path.join(HERE, "rhd_oracle.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-shared",
           "-fPIC", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        ref = orc.lib()  # same C ABI: copy the oracle's signatures
        for name in ("orc_subcycles", "orc_subcycle_box"):
            getattr(L, name).restype = getattr(ref, name).restype
            getattr(L, name).argtypes = getattr(ref, name).argtypes
        L.opc_counts.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        _lib = L
    return _lib


def counted_subcycles(case, n_sub=1):
    """Run n_sub oracle subcycles in the counting build; returns (state, stats, counts dict)."""
    L = lib()
    L.opc_reset()
    saved = orc._lib
    orc._lib = L  # route the wrapper's call through the counting build
    try:
        state, st = orc.subcycles(case, n_sub=n_sub)
    finally:
        orc._lib = saved
    out = (ctypes.c_ulonglong * 6)()
    L.opc_counts(out)
    return state, st, dict(zip(CLASSES, (int(v) for v in out)))


def bulk_ops_per_cell(make_case, sizes=(12, 16, 20, 24, 32)):
    """Cubic fit of the per-class counts of one subcycle over cubic grids N^3, N in `sizes`;
    returns {class: N^3 coefficient} (operations per interior cell-update)."""
    rows = []
    for N in sizes:
        _, _, c = counted_subcycles(make_case(N), n_sub=1)
        rows.append([c[k] for k in CLASSES])
    A = np.array([[N ** 3, N ** 2, N, 1.0] for N in sizes], dtype=np.float64)
    y = np.array(rows, dtype=np.float64)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return dict(zip(CLASSES, (float(v) for v in coef[0])))


def main():
    """Write profiles/opcounts.json: bulk operation counts per cell-update of the 3D throughput
    workload (FULL exchange, beta tau on) from the counting build of the oracle."""
    import json
    import sys

    root = os.path.dirname(HERE)
    sys.path.insert(0, root)
    from paper_1306_0010_gb300 import workloads as wl

    sizes = (12, 16, 20, 24, 32)
    r = bulk_ops_per_cell(lambda N: wl.config4(N=N, n_sub=1), sizes)
    out = {"workload": "3D throughput workload (lognormal rho, k = 512 rho, FULL exchange, beta tau on), one "
                       "subcycle", "method": "counting build of the oracle (opcount.cpp), cubic fit over N = "
                       + ", ".join(str(s) for s in sizes) + "; N^3 coefficient",
           "per_cell_update": {k: round(v, 3) for k, v in r.items()},
           "arith_per_cell_update": round(sum(r[k] for k in ("add", "mul", "div", "sqrt")), 3)}
    path = os.path.join(root, "profiles", "opcounts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
