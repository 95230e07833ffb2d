"""GPU: the split path's error against the FP64 oracle, per configuration that runs it.

For each case the normwise L1 and L-infinity errors of E, F (scaled by max|E| and c max|E|) and T
(scaled by max|T|) are computed against the oracle on the same inputs, printed (run with -s to see
them) beside the split path's bound derived in split_bounds.py, and held to that bound in L-infinity.
Sizes are reduced so the oracle finishes in seconds; the recipes are those of the configurations."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

from split_bounds import split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def norms(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    res = {}
    for k, s in (("E", sE), ("Fx", desc["c"] * sE), ("Fy", desc["c"] * sE), ("Fz", desc["c"] * sE)):
        d = np.abs(out[k] - ref[k]) / s
        res[k] = (float(np.mean(d)), float(np.max(d)))
    if desc["exchange"] == "full":
        d = np.abs(out["T"] - ref["T"]) / float(np.max(np.abs(ref["T"])))
        res["T"] = (float(np.mean(d)), float(np.max(d)))
    return res


def run(rhd, case, n_sub):
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(n_sub, case["chat"], case["dt"])
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    assert g.get_stats()["n_nonfinite"] == 0
    g.close()
    return out


CASES = [
    ("config3 (shell, point source, FULL, beta tau) 64^3 x 25", lambda: wl.config3(N=64, n_sub=25), 25),
    ("config4 (lognormal rho, FULL, beta tau) 64^3 x 20", lambda: wl.config4(N=64, n_sub=20, precision="split"), 20),
]


@pytest.mark.parametrize("name,make,n_sub", CASES, ids=["config3", "config4"])
def test_split_error_report(rhd, name, make, n_sub):
    case = make()
    case["desc"] = dict(case["desc"], precision="split")
    out = run(rhd, case, n_sub)
    ref, _ = orc.subcycles(case, n_sub=n_sub)
    res = norms(out, ref, case["desc"])
    bound = split_bound(case, n_sub)
    print(f"\n{name}: bound {bound:.2e}; " + ", ".join(f"{k} L1 {l1:.2e} Linf {li:.2e}" for k, (l1, li) in res.items()))
    assert max(li for _, li in res.values()) <= bound, res


def test_split_error_report_ensemble(rhd):
    cases = wl.config5(n_grids=3, sizes=(32, 48), n_sub=20, precision="split", seed_offset=90)
    ens = rhd.Ensemble([c["desc"] for c in cases])
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    ens.subcycle(20, 1.0, [c["dt"] for c in cases])
    worst = 0.0
    bound = min(split_bound(c, 20) for c in cases)
    for i, c in enumerate(cases):
        out = ens.get_moments(i)
        out["T"] = ens.get_gas_state(i)
        ref, _ = orc.subcycles(c, n_sub=20)
        res = norms(out, ref, c["desc"])
        print(f"\nconfig5 grid {i} (N={c['desc']['n'][0]}) x 20: " +
              ", ".join(f"{k} L1 {l1:.2e} Linf {li:.2e}" for k, (l1, li) in res.items()))
        worst = max(worst, max(li for _, li in res.values()))
    ens.close()
    assert worst <= bound, (worst, bound)
