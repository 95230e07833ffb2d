"""The option of Section 3.1 step 2: the stiff exchange S_i integrated once per gas step over
Delta t_gas (oracle/gas.py gas_exchange), against closed forms, and the whole cycle with it against the
cycle that exchanges in every subcycle (the two placements differ at first order in the step)."""
import numpy as np
import pytest

from oracle import gas as ogas
from oracle_cycles import run_cycles
from paper_1306_0010_gb300 import workloads as wl


def cell_case(n=(6, 4, 3), seed=3):
    case = wl.gas_case("xchg", n, exchange="full", kappa=5.0, kappa_rho_pow=1, seed=seed)
    f = case["fields"]
    gas = {k: f[k] for k in ("rho", "vx", "vy", "vz", "T")}
    rad = {k: f[k] for k in ("E", "Fx", "Fy", "Fz")}
    return case["desc"], gas, rad, case["chat"]


def total_energy(desc, gas, rad, chat):
    # e + (c / chat) E: what the exchange conserves (Eq. source:energyexchange with chat in the radiation row)
    e = gas["rho"] * gas["T"] / desc["mu_over_kB"] / (desc["gamma"] - 1.0)
    return e + desc["c"] / chat * rad["E"]


def test_exchange_conserves_the_energy_sum_in_every_cell():
    desc, gas, rad, chat = cell_case()
    g1, r1, _ = ogas.gas_exchange(desc, gas, rad, 0.05, chat)
    before, after = total_energy(desc, gas, rad, chat), total_energy(desc, g1, r1, chat)
    assert np.allclose(after, before, rtol=1e-12, atol=0)
    assert not np.allclose(g1["T"], gas["T"])  # it did exchange


def test_equilibrium_cells_are_unchanged():
    desc, gas, rad, chat = cell_case()
    rad = dict(rad, E=desc["a_rad"] * gas["T"] ** 4)
    g1, r1, _ = ogas.gas_exchange(desc, gas, rad, 0.05, chat)
    assert np.allclose(g1["T"], gas["T"], rtol=1e-12, atol=0)
    assert np.allclose(r1["E"], rad["E"], rtol=1e-12, atol=0)


def test_a_long_step_lands_on_the_equilibrium_root():
    # theta = 1 and dt k c >> 1: the backward-Euler step reaches the state with a_R T^4 = E and the same
    # energy sum, i.e. the positive root of (a_R (c/chat)) T^4 + rho T / (mu (gamma - 1)) = sum
    desc, gas, rad, chat = cell_case()
    g1, r1, _ = ogas.gas_exchange(desc, gas, rad, 1e9, chat)
    S = total_energy(desc, gas, rad, chat)
    c, aR = desc["c"], desc["a_rad"]
    for i in np.ndindex(S.shape):
        lin = gas["rho"][i] / desc["mu_over_kB"] / (desc["gamma"] - 1.0)
        roots = np.roots([aR * c / chat, 0.0, 0.0, lin, -S[i]])
        T = max(r.real for r in roots if abs(r.imag) < 1e-9 * abs(r) and r.real > 0)
        assert g1["T"][i] == pytest.approx(T, rel=1e-10)
        assert r1["E"][i] == pytest.approx(aR * T ** 4, rel=1e-9)


def test_flux_is_rescaled_when_the_exchange_drops_E_below_F_over_c():
    desc, gas, rad, chat = cell_case()
    rad = dict(rad, E=np.full_like(rad["E"], 10.0), Fx=np.full_like(rad["E"], 0.99 * desc["c"] * 10.0))
    gas = dict(gas, T=np.full_like(gas["T"], 0.1))  # cold gas absorbs radiation energy
    g1, r1, _ = ogas.gas_exchange(desc, gas, rad, 1.0, chat)
    G = np.sqrt(r1["Fx"] ** 2 + r1["Fy"] ** 2 + r1["Fz"] ** 2) / desc["c"]
    assert np.all(G <= r1["E"] * (1 + 1e-14))
    assert np.all(r1["E"] < 10.0)


def test_exchange_per_gas_step_and_per_subcycle_converge_together():
    """One exchange over Delta t_gas before the gas step, or one in every subcycle: the same equations
    split differently, so the two whole-cycle results differ at first order in Delta t_gas."""
    case = wl.gas_case("xchg_cycle", (24, 1, 1), bc="periodic", exchange="full", kappa=2.0, kappa_rho_pow=1,
                       seed=5, with_v=True, n_sub=4)
    t_end = 0.04
    diffs = []
    for dt in (0.01, 0.005, 0.0025):
        a, ra, _ = run_cycles(case, t_end, dt_fixed=dt)
        b, rb, _ = run_cycles(case, t_end, dt_fixed=dt, exchange_on_gas_step=True)
        diffs.append(max(float(np.max(np.abs(a["T"] - b["T"]) / np.max(a["T"]))),
                         float(np.max(np.abs(ra["E"] - rb["E"]) / np.max(ra["E"])))))
    assert diffs[0] > 1e-6
    assert 1.6 < diffs[0] / diffs[1] < 2.6 and 1.6 < diffs[1] / diffs[2] < 2.6, diffs
