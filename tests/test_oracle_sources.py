"""Pins of the oracle's source-term updates (Section 3.4) against closed forms, invariants and
library root finding.  CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl


def test_theta_factor_orders():
    """theta = 1/2 is the trapezoidal rule (error ~ x^3/12 against exp(-x)); theta = 1 is backward
    Euler (error ~ x^2/2); Eqs. (source:stiff:radmomentum:soln) and the text after it."""
    for x in (1e-2, 3e-3, 1e-3):
        e = math.exp(-x)
        assert orc.theta_factor(0.5, x) - e == pytest.approx(-x ** 3 / 12, rel=2e-2)
        assert orc.theta_factor(1.0, x) - e == pytest.approx(x ** 2 / 2, rel=2e-2)
    # theta = 1 is unconditionally stable: factor in (0, 1] for any x >= 0
    xs = np.logspace(-8, 8, 200)
    f = np.array([orc.theta_factor(1.0, x) for x in xs])
    assert np.all((f > 0) & (f <= 1)) and np.all(np.diff(f) < 0)
    # theta = 0.51 flips sign for x > 1/0.49 (the ringing the paper warns about)
    assert orc.theta_factor(0.51, 3.0) < 0 < orc.theta_factor(0.51, 1.9)


def test_quartic_root_against_numpy_roots():
    g = np.random.default_rng(11)
    for _ in range(4000):
        c4 = 10 ** g.uniform(-6, 6)
        c1 = 1.0 + 10 ** g.uniform(-6, 4)
        c0 = -(10 ** g.uniform(-6, 6))
        x = orc.quartic_root(c4, c1, c0)
        b = min(abs(c0 / c1), abs(c0 / c4) ** 0.25)
        assert 0.0 <= x <= b * (1 + 1e-15)
        r = np.roots([c4, 0.0, 0.0, c1, c0])
        r = r[np.abs(r.imag) < 1e-8 * np.abs(r)].real
        r = r[r > 0]
        assert len(r) == 1  # strictly increasing on x > 0: a single positive root
        # polish numpy's root with two Newton steps before comparing
        y = r[0]
        for _ in range(2):
            y -= (c4 * y ** 4 + c1 * y + c0) / (4 * c4 * y ** 3 + c1)
        assert x == pytest.approx(y, rel=4e-15)


def _desc(theta=1.0, c=10.0):
    return wl.base_desc((1, 1, 1), (1.0, 1.0, 1.0), c=c, exchange="full", theta_F=theta, theta_E=theta,
                        gamma=5.0 / 3.0, mu_over_kB=1.0, a_rad=1.0)


def _e(rho, T, desc):
    return rho * T / desc["mu_over_kB"] / (desc["gamma"] - 1.0)


def test_exchange_conserves_combined_energy():
    """Ebar = e + (c/chat) E is invariant over the exchange (Eq. source:combinedenergy)."""
    g = np.random.default_rng(12)
    for theta in (1.0, 0.51):
        desc = _desc(theta)
        for _ in range(3000):
            chat = 10 ** g.uniform(-1, 0)
            rho, T = math.exp(g.normal()), math.exp(0.3 * g.normal())
            E = desc["a_rad"] * T ** 4 * math.exp(0.5 * g.normal())
            kP, dt = 10 ** g.uniform(-3, 3), 10 ** g.uniform(-4, -1)
            E1, T1, _ = orc.exchange_full(desc, chat, dt, rho, kP, E, T)
            eb0 = _e(rho, T, desc) + (desc["c"] / chat) * E
            eb1 = _e(rho, T1, desc) + (desc["c"] / chat) * E1
            assert eb1 == pytest.approx(eb0, rel=1e-14)


def test_exchange_fixed_point_and_monotone_backward_euler():
    g = np.random.default_rng(13)
    desc = _desc(1.0)
    for _ in range(2000):
        chat = 1.0
        rho, T = math.exp(g.normal()), math.exp(0.3 * g.normal())
        kP, dt = 10 ** g.uniform(-3, 3), 10 ** g.uniform(-4, -1)
        # radiative equilibrium a_R T^4 = E is stationary
        E_eq = desc["a_rad"] * T ** 4
        E1, T1, _ = orc.exchange_full(desc, chat, dt, rho, kP, E_eq, T)
        assert E1 == pytest.approx(E_eq, rel=1e-12) and T1 == pytest.approx(T, rel=1e-12)
        # backward Euler keeps the sign of the departure a_R T^4 - E and shrinks it
        E = E_eq * math.exp(0.7 * g.normal())
        E1, T1, _ = orc.exchange_full(desc, chat, dt, rho, kP, E, T)
        y0 = desc["a_rad"] * T ** 4 - E
        y1 = desc["a_rad"] * T1 ** 4 - E1
        assert y0 * y1 >= 0 and abs(y1) <= abs(y0) * (1 + 1e-12)


def test_exchange_linearised_rate():
    """Near equilibrium y = a_R T^4 - E obeys dy/dt = -chat kP (1 + 4 (c/chat) alpha e^3) y
    (linearising Eqs. source:energyexchange); one theta step multiplies y by
    [1 - (1-theta) lam dt]/[1 + theta lam dt] up to O(y)."""
    for theta in (1.0, 0.51):
        desc = _desc(theta)
        c, chat = desc["c"], 2.0
        rho, T, kP, dt = 1.7, 1.3, 3.0, 0.01
        q = (desc["gamma"] - 1.0) * desc["mu_over_kB"] / rho
        alpha = desc["a_rad"] * q ** 4
        e = _e(rho, T, desc)
        lam = chat * kP * (1.0 + 4.0 * (c / chat) * alpha * e ** 3)
        expect = (1 - (1 - theta) * lam * dt) / (1 + theta * lam * dt)
        for delta in (1e-4, 1e-5):
            E = desc["a_rad"] * T ** 4 * (1 - delta)
            E1, T1, fb = orc.exchange_full(desc, chat, dt, rho, kP, E, T)
            assert fb == 0
            ratio = (desc["a_rad"] * T1 ** 4 - E1) / (desc["a_rad"] * T ** 4 - E)
            assert ratio == pytest.approx(expect, rel=20 * delta)


def test_exchange_theta_fallback_when_unbracketed():
    """For theta < 1 and a stiff step far from equilibrium c0 > 0 and no feasible root exists
    (Section 3.4); the oracle then redoes the step with theta = 1."""
    desc = _desc(0.51)
    rho, T, kP, dt, chat = 1.0, 3.0, 1e3, 1.0, 1.0
    E = 1e-6
    E1, T1, fb = orc.exchange_full(desc, chat, dt, rho, kP, E, T)
    assert fb == 1
    d1 = dict(desc, theta_E=1.0, theta_F=1.0)
    E2, T2, fb2 = orc.exchange_full(d1, chat, dt, rho, kP, E, T)
    assert fb2 == 0 and (E1, T1) == (E2, T2)


def _uniform_case(mode, theta=0.51, beta_tau=False, n=(5, 4, 3)):
    desc = wl.base_desc(n, tuple(1.0 / v for v in n), bc="periodic", c=3.0, exchange=mode,
                        kappa_P=4.0, kappa_F=7.0, kappa_rho_pow=0, theta_F=theta, theta_E=theta,
                        beta_tau=beta_tau)
    shp = (n[2], n[1], n[0])
    fields = {"E": np.full(shp, 1.3), "Fx": np.full(shp, 0.9), "Fy": np.full(shp, -0.6), "Fz": np.full(shp, 0.3),
              "T": np.full(shp, 1.1), "rho": np.full(shp, 0.8), "vx": None, "vy": None, "vz": None,
              "kP": None, "kF": None, "j": None}
    chat = 2.0
    return {"name": "uniform", "desc": desc, "fields": fields, "chat": chat, "dt": wl.cfl_dt(desc, chat), "n_sub": 1}


@pytest.mark.parametrize("mode", ["absorb", "frozen_t", "equilibrium"])
def test_uniform_state_is_pure_theta_decay(mode):
    """A uniform periodic state has no transport; one subcycle applies exactly the factor of Eq.
    (source:stiff:radmomentum:soln) to F over the full dt, and by mode Eq. (source:stiff:radenergy:soln)
    or the frozen-temperature theta update to E."""
    case = _uniform_case(mode)
    out, st = orc.subcycles(case)
    d, chat, dt = case["desc"], case["chat"], case["dt"]
    xF = chat * d["kappa_F"] * dt
    xP = chat * d["kappa_P"] * dt
    fF = orc.theta_factor(d["theta_F"], xF)
    for k in ("Fx", "Fy", "Fz"):
        F0 = case["fields"][k][0, 0, 0]
        # F -> G = F/c -> G * fF -> F = c * G: at most one rounding per step
        assert np.allclose(out[k], (F0 / d["c"]) * fF * d["c"], rtol=2.3e-16, atol=0)
    E0 = case["fields"]["E"][0, 0, 0]
    if mode == "absorb":
        expect = E0 * orc.theta_factor(d["theta_E"], xP)
    elif mode == "frozen_t":
        th, T = d["theta_E"], 1.1
        expect = (E0 * (1 - (1 - th) * xP) + xP * d["a_rad"] * T ** 4) / (1 + th * xP)
    else:
        expect = E0
    assert np.allclose(out["E"], expect, rtol=4.5e-16, atol=0)
    assert st["n_realizability_fix"] == 0 and st["n_nonfinite"] == 0


def test_beta_tau_flux_relaxes_to_comoving_value():
    """With the O(beta tau) terms (Eq. m1:simplifiedsource) a uniform medium moving at v drives
    G = F/c towards (4/3) E v / c, radiation carried along with the gas (the dynamic-diffusion
    balance of -chat kF G and chat (4/3) kF E v/c); meanwhile E changes only through
    chat kF (v/c).G, which is positive and second order in v/c."""
    n = (4, 3, 3)
    desc = wl.base_desc(n, tuple(1.0 / v for v in n), bc="periodic", c=100.0, exchange="equilibrium",
                        beta_tau=True, kappa_P=50.0, kappa_F=50.0, kappa_rho_pow=0, theta_F=1.0, theta_E=1.0)
    shp = (n[2], n[1], n[0])
    v = np.array([0.7, -0.4, 0.2])
    fields = {"E": np.full(shp, 2.0), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
              "T": np.ones(shp), "rho": np.ones(shp), "vx": np.full(shp, v[0]), "vy": np.full(shp, v[1]),
              "vz": np.full(shp, v[2]), "kP": None, "kF": None, "j": None}
    chat = 1.0
    case = {"desc": desc, "fields": fields, "chat": chat, "dt": wl.cfl_dt(desc, chat), "n_sub": 400}
    out, st = orc.subcycles(case)
    E1 = out["E"][0, 0, 0]
    G1 = np.array([out[k][0, 0, 0] for k in ("Fx", "Fy", "Fz")]) / desc["c"]
    # G trails the slowly growing E by O(growth / (chat kF)) ~ 1e-4
    assert np.allclose(G1, (4.0 / 3.0) * E1 * v / desc["c"], rtol=1e-3)
    beta2 = float(v @ v) / desc["c"] ** 2
    t = case["n_sub"] * case["dt"]
    # dE/dt = chat kF (4/3) E beta^2 once G has relaxed (relaxation time 1/(chat kF) << t)
    growth = math.log(E1 / 2.0) / t
    assert growth == pytest.approx(chat * 50.0 * (4.0 / 3.0) * beta2, rel=0.05)
