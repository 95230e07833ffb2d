"""GPU: the split path's stiff sources in FP64, on stiff exchanges whose gas energy is far above the
radiation's (K = e / ((c/chat) E) up to 2e4; Section 3.4, Eqs. source:energyupdate - source:polynomial
and the condition number of Eq. source:kappacond).

Uniform states: every cell holds the same state, so the FP32 transport of each subcycle cancels
exactly (equal fluxes on all faces) and only the stiff sources act.  The split path must then meet
the FP64 path's bound (1e-12 normwise against the oracle) on every kernel that runs it: the two-pass
pair (3D), the fused kernel (1D, 2D, 3D) and both ensemble variants; for FULL (theta = 1 and 0.51),
ABSORB and FROZEN_T.  An FP32 theta factor or exchange would miss it by orders of magnitude.

Non-uniform states: the split bound derived in split_bounds.py, which does not grow with K."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

from split_bounds import gas_energy_ratio, split_bound

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


def errors(out, ref, desc, with_T):
    sE = float(np.max(np.abs(ref["E"])))
    e = {"E": float(np.max(np.abs(out["E"] - ref["E"]))) / sE}
    for k in ("Fx", "Fy", "Fz"):
        e[k] = float(np.max(np.abs(out[k] - ref[k]))) / (desc["c"] * sE)
    if with_T:
        e["T"] = float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(np.abs(ref["T"])))
    return e


def run(rhd, case, flags=0, launch=None):
    g = rhd.Grid(dict(case["desc"], flags=flags))
    if launch is not None:
        g.set_launch_config(launch)
    g.load_case(case)
    g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    st = g.get_stats()
    g.close()
    return out, st


UNIFORM = [
    ("3d_full", (12, 10, 9), dict(exchange="full")),
    ("3d_full_theta051", (12, 10, 9), dict(exchange="full", theta=0.51)),
    ("3d_absorb_theta051", (12, 10, 9), dict(exchange="absorb", theta=0.51)),
    ("3d_frozen_t", (12, 10, 9), dict(exchange="frozen_t")),
    ("2d_full", (24, 20, 1), dict(exchange="full")),
    ("1d_full", (40, 1, 1), dict(exchange="full", K=2.0e3)),
    ("3d_full_radiation_dominated", (12, 10, 9), dict(exchange="full", K=1e-3, rho0=1.0)),
]


@pytest.mark.parametrize("flags", [0, 2], ids=["twopass", "fused"])
@pytest.mark.parametrize("name,n,kw", UNIFORM, ids=[u[0] for u in UNIFORM])
def test_uniform_stiff_split_meets_fp64_bound(rhd, name, n, kw, flags):
    if flags and n[2] == 1:
        pytest.skip("1D and 2D split grids always run the fused kernel")
    case = wl.stiff_case(name, n, uniform=True, n_sub=12, **kw)
    out, st = run(rhd, case, flags=flags)
    ref, rst = orc.subcycles(case)
    e = errors(out, ref, case["desc"], case["desc"]["exchange"] == "full")
    print(f"\n{name} (K = {gas_energy_ratio(case):.3g}): " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert max(e.values()) <= FP64_TOL, e
    assert st["n_nonfinite"] == 0
    assert st["n_theta_fallback"] == rst["n_theta_fallback"]
    # the state stays uniform: every cell took the same steps
    for k in ("E", "Fx", "T"):
        assert np.ptp(out[k]) == 0.0, k


@pytest.mark.parametrize("flags", [0, 2], ids=["twopass", "fused"])
def test_uniform_stiff_split_ensemble(rhd, flags):
    cases = [wl.stiff_case(f"ens{i}", (n, n, n), uniform=True, n_sub=8, K=K)
             for i, (n, K) in enumerate(((8, 2e4), (12, 50.0), (16, 2e3)))]
    # one chat for the ensemble; each grid its own dt and opacity
    ens = rhd.Ensemble([dict(c["desc"], flags=flags) for c in cases])
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    ens.subcycle(8, 1.0, [c["dt"] for c in cases])
    assert ens.get_stats()["n_nonfinite"] == 0
    for i, c in enumerate(cases):
        out = ens.get_moments(i)
        out["T"] = ens.get_gas_state(i)
        ref, _ = orc.subcycles(c, n_sub=8)
        e = errors(out, ref, c["desc"], True)
        assert max(e.values()) <= FP64_TOL, (i, e)
    ens.close()


NONUNIFORM = [
    ("3d_K2e4", (20, 13, 11), dict(K=2.0e4)),
    ("3d_K2e4_outflow", (20, 13, 11), dict(K=2.0e4, bc="outflow")),
    ("3d_K50_theta051", (20, 13, 11), dict(K=50.0, theta=0.51)),
    ("2d_K2e4", (33, 17, 1), dict(K=2.0e4)),
]


@pytest.mark.parametrize("flags", [0, 2], ids=["twopass", "fused"])
@pytest.mark.parametrize("name,n,kw", NONUNIFORM, ids=[u[0] for u in NONUNIFORM])
def test_stiff_split_within_derived_bound(rhd, name, n, kw, flags):
    if flags and n[2] == 1:
        pytest.skip("1D and 2D split grids always run the fused kernel")
    n_sub = 10
    case = wl.stiff_case(name, n, uniform=False, n_sub=n_sub, **kw)
    out, st = run(rhd, case, flags=flags)
    ref, _ = orc.subcycles(case)
    e = errors(out, ref, case["desc"], True)
    bound = split_bound(case, n_sub)
    K = gas_energy_ratio(case)
    print(f"\n{name} (K up to {K:.3g}): bound {bound:.2e}; " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert st["n_nonfinite"] == 0
    assert max(e.values()) <= bound, (bound, e)
