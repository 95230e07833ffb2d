"""GPU: the grid reductions behind the reduced-speed-of-light helpers (v_max of Eq. algorithm:ceff,
the domain's optical depth along the axes) against the oracle on the same inputs, and a gas cycle
planned with them."""
import ctypes

import numpy as np
import pytest

from oracle import rsla
from paper_1306_0010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

RTOL = 1e-13  # sums of up to a few hundred terms in another order


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


CASES = [
    dict(n=(20, 12, 10), with_v=True, kP_array=False, precision="split"),
    dict(n=(37, 5, 9), with_v=True, kP_array=True, precision="fp64"),
    dict(n=(64, 1, 1), with_v=False, kP_array=False, precision="fp64"),
    dict(n=(33, 17, 1), with_v=True, kP_array=True, precision="fp64"),
]


@pytest.mark.parametrize("spec", CASES, ids=lambda s: "x".join(map(str, s["n"])))
def test_reductions_match_oracle(rhd, spec):
    case = wl.parity_case("rsla", spec["n"], bc="outflow", exchange="full", beta_tau=spec["with_v"],
                          with_v=spec["with_v"], kappa=40.0, kP_array=spec["kP_array"], n_sub=3, seed=61,
                          precision=spec["precision"])
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    for step in range(2):
        # the current T and E (the FULL exchange changes both) read back as the oracle's inputs
        T = g.get_gas_state()
        E = g.get_moments()["E"]
        fields = dict(case["fields"], T=T)
        v_ref = rsla.max_signal_speed(case["desc"], fields, E)
        tau_ref = rsla.max_optical_depth(case["desc"], fields)
        assert g.max_signal_speed() == pytest.approx(v_ref, rel=RTOL, abs=0)
        assert g.max_optical_depth() == pytest.approx(tau_ref, rel=RTOL, abs=0)
        g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    g.close()


def test_plan_a_gas_cycle(rhd):
    """chat from the static-diffusion criterion, then the subcycles that span dt_gas: the step passes
    the library's CFL check and advances the grid."""
    case = wl.parity_case("plan", (24, 16, 12), bc="periodic", exchange="full", kappa=5.0, c=1000.0, n_sub=1,
                          seed=62, precision="split")  # static gas: v_max is the effective sound speed
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    v_max, tau_max = g.max_signal_speed(), g.max_optical_depth()
    chat = rhd.suggest_chat(case["desc"]["c"], v_max, tau_max, ratio=10.0)
    assert chat == rsla.suggest_chat(case["desc"]["c"], v_max, tau_max, 10.0)
    dx = min(case["desc"]["dx"])
    dt_gas, dt_rad, n_sub = rhd.time_steps(case["desc"]["cfl"], dx, v_max, chat)
    assert n_sub >= 10 and abs(n_sub * dt_rad - dt_gas) <= 1e-12 * dt_gas
    g.radiation_subcycle(n_sub, chat, dt_rad)
    st = g.get_stats()
    assert st["n_subcycles"] == n_sub and st["n_nonfinite"] == 0
    g.close()


def test_errors(rhd):
    case = wl.parity_case("rsla_err", (16, 8, 8), n_sub=1, seed=63, precision="split")
    g = rhd.Grid(case["desc"])
    with pytest.raises(rhd.RhdError) as ei:
        g.max_optical_depth()  # gas state not set
    assert ei.value.status == rhd.ERR_STATE
    f = case["fields"]
    g.set_gas_state(f["rho"], f["T"])
    with pytest.raises(rhd.RhdError) as ei:
        g.max_signal_speed()  # moments not set
    assert ei.value.status == rhd.ERR_STATE
    assert g.max_optical_depth() > 0
    # a zero density makes c_eff = sqrt(0 / 0) NaN: reported, and the context stays usable
    rho = f["rho"].copy()
    rho[3, 4, 5] = 0.0
    g.set_gas_state(rho, f["T"])
    g.set_moments(f["E"], f["Fx"], f["Fy"], f["Fz"])
    with pytest.raises(rhd.RhdError) as ei:
        g.max_signal_speed()
    assert ei.value.status == rhd.ERR_NONFINITE
    g.set_gas_state(f["rho"], f["T"])
    assert np.isfinite(g.max_signal_speed())
    g.close()
    ens = rhd.Ensemble([case["desc"]])
    ens.load_case(0, case)
    out = ctypes.c_double()
    assert rhd.lib().rhd_max_signal_speed(ens._ctx, ctypes.byref(out)) == rhd.ERR_STATE
    assert rhd.lib().rhd_max_optical_depth(ens._ctx, ctypes.byref(out)) == rhd.ERR_STATE
    ens.close()
