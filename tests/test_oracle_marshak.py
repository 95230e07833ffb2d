"""The oracle's pieces of the non-equilibrium Marshak wave (Section 4.1.4) against what mathematics and
physics fix: the linear (Pomraning) exchange conserves v / (eps c) + E / chat and relaxes v - E by the
theta-scheme factor of a linear ODE (hence to exp(-lambda t) under refinement), and the Su & Olson
surface value starts at 0 on the cold medium, rises monotonically and tends to 1 (F -> 0 in the
equilibrium diffusion limit), with the boundary state meeting c E + 2 F = 4 F_inc."""
import math

import numpy as np
import pytest

from oracle import marshak, oracle as orc
from paper_1306_0010_gb300 import workloads as wl


def desc(eps=1.0, theta=1.0, c=1.0, a=1.0):
    d = wl.base_desc((8, 1, 1), (0.1, 1.0, 1.0), c=c, exchange="linear", theta_E=theta)
    d["a_rad"] = a
    d["linear_eps"] = eps
    return d


@pytest.mark.parametrize("eps,chat,theta", [(1.0, 1.0, 1.0), (0.3, 1.0, 0.5), (2.0, 0.25, 1.0), (0.7, 0.1, 0.51)])
def test_linear_exchange_conserves_and_matches_the_linear_theta_scheme(eps, chat, theta):
    c, a, kP, dt = 1.0, 1.7, 3.0, 0.05
    d = desc(eps, theta, c, a)
    E, T = 0.3, 1.2
    v = a * T ** 4
    lam = (eps * c + chat) * kP
    E1, T1 = orc.exchange_linear(d, chat, dt, kP, E, T)
    v1 = a * T1 ** 4
    # the conserved combination of dv/dt = -eps c kP (v - E), dE/dt = chat kP (v - E)
    assert v1 / (eps * c) + E1 / chat == pytest.approx(v / (eps * c) + E / chat, rel=1e-14)
    # w = v - E obeys dw/dt = -lambda w; the theta scheme multiplies it by [1 - (1-theta) lambda dt] / [1 + theta lambda dt]
    assert (v1 - E1) == pytest.approx((v - E) * (1 - (1 - theta) * lam * dt) / (1 + theta * lam * dt), rel=1e-12)


def test_linear_exchange_converges_to_the_exact_relaxation():
    eps, chat, c, a, kP, t = 0.5, 0.8, 1.0, 1.0, 2.0, 0.7
    d = desc(eps, 0.5, c, a)
    E0, T0 = 2.0, 0.5
    w0 = a * T0 ** 4 - E0
    lam = (eps * c + chat) * kP
    errs = []
    for n in (50, 100, 200):
        E, T = E0, T0
        for _ in range(n):
            E, T = orc.exchange_linear(d, chat, t / n, kP, E, T)
        errs.append(abs((a * T ** 4 - E) - w0 * math.exp(-lam * t)))
    # Crank-Nicolson (theta = 1/2) is second order
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_linear_exchange_on_a_grid_is_the_cell_exchange():
    """No flux, uniform state, periodic: transport vanishes and every cell follows the single-cell update."""
    n = 16
    d = desc(1.3, 1.0, 1.0, 1.0)
    d["n"], d["dx"] = (n, 1, 1), (1.0 / n, 1.0, 1.0)
    d["bc_lo"] = d["bc_hi"] = ["periodic"] * 3
    d["kappa_P"] = d["kappa_F"] = 5.0
    d["kappa_rho_pow"] = 1
    shp = (1, 1, n)
    f = {"E": np.full(shp, 0.2), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp), "T": np.full(shp, 0.9),
         "rho": np.full(shp, 1.0), "vx": None, "vy": None, "vz": None, "kP": None, "kF": None, "j": None}
    case = {"desc": d, "fields": f, "chat": 1.0, "dt": 0.01, "n_sub": 5}
    st, _ = orc.subcycles(case)
    E, T = 0.2, 0.9
    for _ in range(5):
        E, T = orc.exchange_linear(d, 1.0, 0.01, 5.0, E, T)
    assert np.allclose(st["E"], E, rtol=1e-14, atol=0) and np.allclose(st["T"], T, rtol=1e-14, atol=0)


def test_surface_value_limits_and_monotonicity():
    eps = 1.0
    taus = [0.01, 0.03, 0.1, 0.3, 1.0, 3.0, 10.0, 30.0, 100.0, 1000.0]
    u = [marshak.surface_u(t, eps) for t in taus]
    assert all(a < b for a, b in zip(u, u[1:]))
    assert 0.0 < u[0] and u[-1] < 1.0
    assert marshak.surface_u(1e5, eps) > 0.995
    # at tau = 0 the two integrals cancel the 1 exactly (cold surface): the midpoint sums tend to 0
    z = [marshak.surface_u(0.0, eps, n) for n in (1024, 4096, 16384, 65536)]
    assert all(b < a for a, b in zip(z, z[1:])) and z[-1] < 1e-3
    # the midpoint rule has converged where the integrands are smooth (tau > 0)
    for t in (0.1, 1.0, 10.0):
        assert marshak.surface_u(t, eps, 4096) == pytest.approx(marshak.surface_u(t, eps, 65536), abs=1e-6)


def test_boundary_state_meets_the_marshak_condition():
    for tau in (0.1, 1.0, 10.0):
        E, F = marshak.boundary_state(tau, 1.0, 0.25, 1.0)
        assert 1.0 * E + 2.0 * F == pytest.approx(4 * 0.25, rel=1e-15)
        assert E > 0 and F > 0
