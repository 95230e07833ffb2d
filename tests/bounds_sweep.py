"""Tiny and ragged grids through the bounds-checked library (librhd_debug.so), one JSON line per case:
the out-of-range index count of the kernels' checks and the normwise error against the oracle.

Run by tests/test_gpu_bounds.py in a separate process (the binding loads one library per process)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_1306_0010_gb300 import rhd, workloads as wl  # noqa: E402
from split_bounds import split_bound  # noqa: E402

D = {"dirichlet": ([[1.2, 0.3, 0.0, 0.0], [0.9, 0.0, 0.2, 0.0], [1.1, 0.0, 0.0, 0.4]],
                   [[0.8, -0.2, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0], [0.7, 0.0, 0.0, -0.1]])}

CASES = [
    # (n, bc, precision, launch) ; launch None = the default configuration
    ((5, 3, 3), "periodic", "split", None),
    ((4, 3, 3), "periodic", "fp64", None),
    ((5, 3, 3), (["outflow", "reflect", "dirichlet"], ["dirichlet", "outflow", "reflect"]), "split", None),
    ((5, 3, 3), (["outflow", "reflect", "dirichlet"], ["dirichlet", "outflow", "reflect"]), "fp64", None),
    ((3, 4, 5), "reflect", "split", None),
    ((7, 1, 1), "outflow", "split", None),
    ((7, 1, 1), "periodic", "fp64", None),
    ((5, 3, 1), (["periodic", "dirichlet", "periodic"], ["periodic", "outflow", "periodic"]), "split", None),
    ((37, 11, 7), "periodic", "split", {"variant": "twopass", "tile": (32, 8), "z_chunk": 16, "staging": "cpasync"}),
    ((37, 11, 7), "outflow", "split", {"variant": "twopass", "tile": (32, 8), "z_chunk": 16, "staging": "tma"}),
    ((33, 9, 5), (["reflect", "periodic", "outflow"], ["outflow", "periodic", "reflect"]), "split",
     {"variant": "fused", "tile": (32, 8), "z_chunk": 32, "staging": "cpasync"}),
    ((33, 9, 5), "outflow", "split", {"variant": "fused", "tile": (64, 8), "z_chunk": 32, "staging": "cpasync"}),
    ((19, 13, 11), "outflow", "fp64", {"variant": "fused", "tile": (16, 16), "z_chunk": 8, "staging": "cpasync"}),
    ((9, 4, 3), "outflow", "split", None),
    ((33, 9, 5), "outflow", "split", {"variant": "twopass", "tile": (32, 8), "z_chunk": 3, "staging": "cpasync"}),
]


def errors(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    e = [float(np.max(np.abs(out["E"] - ref["E"]))) / sE]
    e += [float(np.max(np.abs(out[k] - ref[k]))) / (desc["c"] * sE) for k in ("Fx", "Fy", "Fz")]
    e.append(float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(np.abs(ref["T"]))))
    return max(e)


def stats_or_status(get):
    try:
        return get(), rhd.OK, ""
    except rhd.RhdError as err:
        return None, err.status, str(err)


def main():
    rhd.lib(rhd.DEBUG_LIB_PATH)
    print(json.dumps({"bounds_checked": int(rhd.lib().rhd_bounds_checked())}), flush=True)
    for i, (n, bc, precision, launch) in enumerate(CASES):
        dirichlet = D["dirichlet"] if "dirichlet" in json.dumps(bc) else None
        # with_j alternates: the per-cell emissivity array switches the kernels' optional-array paths
        case = wl.parity_case("bounds", n, bc=bc, exchange="full", beta_tau=True, with_j=i % 2 == 0, n_sub=2,
                              seed=90 + i, precision=precision, dirichlet=dirichlet, kP_array=i % 3 == 0)
        g = rhd.Grid(case["desc"])
        if launch is not None:
            g.set_launch_config(launch)
        g.load_case(case)
        g.reset_stats()
        g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
        st, status, msg = stats_or_status(g.get_stats)
        out = g.get_moments()
        out["T"] = g.get_gas_state()
        g.close()
        ref, _ = orc.subcycles(case)
        print(json.dumps({"case": i, "n": n, "precision": precision, "launch": launch and launch["variant"],
                          "status": status, "bounds_violations": None if st is None else st["bounds_violations"],
                          "message": msg, "error": errors(out, ref, case["desc"]),
                          "bound": split_bound(case, case["n_sub"])}), flush=True)
    # an ensemble of tiny grids (persistent kernels, work queue)
    cases = [wl.parity_case("bounds_ens", n, bc="outflow", exchange="full", n_sub=2, seed=120 + k, precision="split")
             for k, n in enumerate([(5, 3, 3), (9, 4, 3), (33, 9, 5)])]
    ens = rhd.Ensemble([c["desc"] for c in cases])
    for k, c in enumerate(cases):
        ens.load_case(k, c)
    ens.reset_stats()
    ens.subcycle(2, 1.0, [c["dt"] for c in cases])
    st, status, msg = stats_or_status(ens.get_stats)
    err = 0.0
    for k, c in enumerate(cases):
        out = ens.get_moments(k)
        out["T"] = ens.get_gas_state(k)
        ref, _ = orc.subcycles(c, n_sub=2)
        err = max(err, errors(out, ref, c["desc"]))
    ens.close()
    print(json.dumps({"case": "ensemble", "precision": "split", "status": status,
                      "bounds_violations": None if st is None else st["bounds_violations"], "message": msg,
                      "error": err, "bound": min(split_bound(c, 2) for c in cases)}), flush=True)


if __name__ == "__main__":
    main()
