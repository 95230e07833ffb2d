"""GPU: states in cgs units, where the split path's FP32 transport and double-float stiff sources must
stay inside the FP32 range (E from 1e-11 to 1e7 erg cm^-3, a_R = 7.6e-15, c = 3e10, mu/k_B = 7.3e-9),
against the oracle: the FP64 path at 1e-12, the split path within its derived bound, on the two-pass
and the fused kernels.  A state beyond the FP32 range, or whose flux chat E overflows it, is reported
as non-finite on split grids (the FP64 path takes it)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

from split_bounds import split_bound

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def errors(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    e = {"E": float(np.max(np.abs(out["E"] - ref["E"]))) / sE}
    for k in ("Fx", "Fy", "Fz"):
        e[k] = float(np.max(np.abs(out[k] - ref[k]))) / (desc["c"] * sE)
    e["T"] = float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(np.abs(ref["T"])))
    return e


def run(rhd, case, flags=0):
    g = rhd.Grid(dict(case["desc"], flags=flags))
    g.load_case(case)
    g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    st = g.get_stats(allow_nonfinite=True)
    g.close()
    return out, st


CASES = [("3d", (16, 12, 10), 0), ("3d_fused", (16, 12, 10), 2), ("2d", (24, 18, 1), 0), ("1d", (48, 1, 1), 0)]


@pytest.mark.parametrize("regime", sorted(wl.PHYSICAL_REGIMES))
@pytest.mark.parametrize("name,n,flags", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_cgs_units_match_the_oracle(rhd, precision, name, n, flags, regime):
    if flags and precision == "fp64":
        pytest.skip("the FP64 path has one kernel")
    case = wl.physical_units_case(f"{regime}_{name}", n, regime, precision=precision, n_sub=4, seed=len(name))
    out, st = run(rhd, case, flags=flags)
    ref, rst = orc.subcycles(case)
    e = errors(out, ref, case["desc"])
    tol = FP64_TOL if precision == "fp64" else split_bound(case, case["n_sub"])
    print(f"\n{precision} {name} {regime}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()) + f" (tol {tol:.1e})")
    assert st["n_nonfinite"] == 0 and st["wait_timeouts"] == 0
    assert st["n_theta_fallback"] == rst["n_theta_fallback"]
    assert max(e.values()) <= tol, e


@pytest.mark.parametrize("flags", [0, 2], ids=["twopass", "fused"])
@pytest.mark.parametrize("what", ["E_beyond_fp32", "flux_beyond_fp32"])
def test_split_state_beyond_fp32_range_is_reported(rhd, what, flags):
    """E = 1e39 erg cm^-3 in one cell is beyond FP32; E = 1e31 fits, but its flux chat E (chat = c/100)
    does not.  The split grid reports either as non-finite; the FP64 grid advances the same state."""
    case = wl.physical_units_case(what, (16, 12, 10), "protostellar_disk", precision="split", n_sub=2, seed=9)
    f = dict(case["fields"])
    for k in ("E", "Fx", "Fy", "Fz"):
        f[k] = f[k].copy()
    f["E"][7, 5, 4] = 1e39 if what == "E_beyond_fp32" else 1e31
    f["Fx"][7, 5, 4] = f["Fy"][7, 5, 4] = f["Fz"][7, 5, 4] = 0.0
    case["fields"] = f
    g = rhd.Grid(dict(case["desc"], flags=flags))
    g.load_case(case)
    g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    with pytest.raises(rhd.RhdError) as ei:
        g.get_stats()
    assert ei.value.status == rhd.ERR_NONFINITE
    g.close()
    fp64 = dict(case, desc=dict(case["desc"], precision="fp64"))
    out, st = run(rhd, fp64)
    assert st["n_nonfinite"] == 0 and np.isfinite(out["E"]).all()
    ref, _ = orc.subcycles(fp64)
    assert max(errors(out, ref, fp64["desc"]).values()) <= FP64_TOL
