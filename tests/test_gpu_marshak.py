"""GPU: the non-equilibrium Marshak wave (Section 4.1.4) through the library, the low x face set before
every subcycle from the Su & Olson surface value, against the oracle run with the same boundary
schedule: the linear (Pomraning) exchange, the time-dependent Dirichlet face and the 1D kernels."""
import copy

import numpy as np
import pytest

from oracle import marshak, oracle as orc
from paper_1306_0010_gb300 import workloads as wl

from split_bounds import split_bound

pytestmark = pytest.mark.gpu

N_QUAD = 1024


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def oracle_run(case, n_sub):
    c = copy.deepcopy(case)
    m = c["marshak"]
    state = None
    for k in range(n_sub):
        tau = m["tau_rate"] * (k + 0.5) * c["dt"]
        E_b, F_b = marshak.boundary_state(tau, m["eps"], m["F_inc"], c["desc"]["c"], N_QUAD)
        c["desc"]["dirichlet_lo"][0] = [E_b, F_b, 0.0, 0.0]
        state, _ = orc.subcycles(c, n_sub=1)
        c["fields"] = dict(c["fields"], E=state["E"], Fx=state["Fx"], Fy=state["Fy"], Fz=state["Fz"], T=state["T"])
    return state


@pytest.mark.parametrize("precision,N,tau,eps", [("fp64", 64, 10.0, 1.0), ("fp64", 100, 3.0, 0.5),
                                                 ("split", 64, 10.0, 1.0)])
def test_marshak_wave_matches_oracle(rhd, precision, N, tau, eps):
    case = wl.marshak_case(N, eps=eps, precision=precision)
    n_sub = wl.marshak_subcycles(tau, case)
    tol = 1e-12 if precision == "fp64" else split_bound(case, n_sub)
    ref = oracle_run(case, n_sub)
    g = rhd.Grid(dict(case["desc"], flags=rhd.FLAG_NO_GRAPH))
    g.load_case(case)
    g.marshak_advance(n_sub, case["chat"], case["dt"], 0.0, case["marshak"], n_quad=N_QUAD)
    out = g.get_moments()
    T = g.get_gas_state()
    st = g.get_stats()
    g.close()
    assert st["n_nonfinite"] == 0 and st["n_subcycles"] == n_sub
    sE = float(np.max(ref["E"]))
    assert float(np.max(np.abs(out["E"] - ref["E"]))) <= tol * sE
    assert float(np.max(np.abs(out["Fx"] - ref["Fx"]))) <= tol * case["desc"]["c"] * sE
    assert float(np.max(np.abs(T - ref["T"]))) <= tol * float(np.max(ref["T"]))
    # the wave has entered the slab: heated near the boundary, cold far away (v = T^4 with a_R = 1)
    assert ref["T"][0, 0, 0] ** 4 > 0.1 and ref["T"][0, 0, -1] ** 4 < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_linear_exchange_3d_grid_and_ensemble(rhd, precision):
    """The linear exchange on 3D grids: a single grid (split grids with it take the fused kernel) and
    an ensemble of two grids, against the oracle."""
    cases = [wl.parity_case(f"lin{i}", n, bc="outflow", exchange="linear", beta_tau=False, kappa=3.0, n_sub=3,
                            seed=150 + i, precision=precision) for i, n in enumerate([(20, 12, 10), (17, 9, 11)])]
    for c in cases:
        c["desc"]["linear_eps"] = 0.6
    refs = [orc.subcycles(c)[0] for c in cases]
    tol = 1e-12 if precision == "fp64" else min(split_bound(c, 3) for c in cases)

    def errors(out, ref, c):
        sE = float(np.max(ref["E"]))
        e = max(float(np.max(np.abs(out[k] - ref[k]))) / (c["desc"]["c"] * sE) for k in ("Fx", "Fy", "Fz"))
        e = max(e, float(np.max(np.abs(out["E"] - ref["E"]))) / sE)
        return max(e, float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(ref["T"])))

    g = rhd.Grid(cases[0]["desc"])
    if precision == "split":
        assert g.launch_config()["variant"] == "fused"
    g.load_case(cases[0])
    g.radiation_subcycle(cases[0]["n_sub"], cases[0]["chat"], cases[0]["dt"])
    out = dict(g.get_moments(), T=g.get_gas_state())
    g.close()
    assert errors(out, refs[0], cases[0]) <= tol
    ens = rhd.Ensemble([c["desc"] for c in cases])
    assert ens.launch_config()["variant"] == "fused"
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    ens.subcycle(3, cases[0]["chat"], [c["dt"] for c in cases])
    for i, c in enumerate(cases):
        out = dict(ens.get_moments(i), T=ens.get_gas_state(i))
        assert errors(out, refs[i], c) <= tol, i
    ens.close()
