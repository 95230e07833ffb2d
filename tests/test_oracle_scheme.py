"""Pins of the oracle's whole subcycle against conservation, closed-form wave solutions,
symmetries and a brute-force re-evaluation.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _dV(desc):
    return float(np.prod([desc["dx"][d] for d in range(3) if desc["n"][d] > 1]))


def _totals(state, desc):
    dV = _dV(desc)
    return np.array([state["E"].sum(), state["Fx"].sum(), state["Fy"].sum(), state["Fz"].sum()]) * dV


# ----------------------------------------------------------------------------- P4 conservation

def test_conservation_periodic():
    case = wl.parity_case("cons", (10, 8, 6), bc="periodic", exchange="equilibrium", kappa=0.0,
                          fmax=0.5, n_sub=20, seed=3)
    before = _totals(case["fields"], case["desc"])
    out, st = orc.subcycles(case)
    after = _totals(out, case["desc"])
    scale = case["fields"]["E"].sum() * _dV(case["desc"])
    assert st["n_realizability_fix"] == 0 and st["n_nonfinite"] == 0
    assert np.all(np.abs(after - before) <= 2e-14 * scale * case["desc"]["c"])


def test_energy_budget_outflow_and_reflect():
    """With outflow faces the change of total E equals the energy that left through them; with
    reflecting faces nothing leaves (mirror states give zero energy flux)."""
    for bc, expect_zero in (("outflow", False), ("reflect", True)):
        case = wl.parity_case("budget", (9, 7, 5), bc=bc, exchange="equilibrium", kappa=0.0, fmax=0.6,
                              n_sub=1, seed=4)
        tot = case["fields"]["E"].sum() * _dV(case["desc"])
        cur = case
        for _ in range(8):
            out, st = orc.subcycles(cur)
            new = out["E"].sum() * _dV(case["desc"])
            assert st["n_realizability_fix"] == 0
            assert new == pytest.approx(tot - st["boundary_E_out"], rel=2e-14)
            if expect_zero:
                assert abs(st["boundary_E_out"]) < 1e-15 * tot
            tot = new
            cur = dict(cur, fields=dict(cur["fields"], **{k: out[k] for k in ("E", "Fx", "Fy", "Fz")}))


# ----------------------------------------------------------------------------- P5 streaming front

def test_free_streaming_front():
    """A beam with F = cE (f = 1) entering an empty, transparent medium through a Dirichlet face
    moves at chat (Section 3.3: all waves travel at chat mu as f -> 1)."""
    N = 128
    desc = wl.base_desc((N, 1, 1), (1.0 / N, 1.0, 1.0), bc=(["dirichlet", "periodic", "periodic"],
                        ["outflow", "periodic", "periodic"]), c=1.0, exchange="equilibrium",
                        E_floor=1e-10, limiter="minmod")
    desc["dirichlet_lo"][0] = [1.0, 1.0, 0.0, 0.0]
    shp = (1, 1, N)
    f = {"E": np.full(shp, 1e-10), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
         "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None, "kP": None,
         "kF": None, "j": None}
    chat = 1.0
    dt = 0.4 / N
    n = 150
    case = {"desc": desc, "fields": f, "chat": chat, "dt": dt, "n_sub": n}
    out, st = orc.subcycles(case)
    E = out["E"][0, 0]
    x = (np.arange(N) + 0.5) / N
    t = n * dt
    front = x[np.argmax(E < 0.5)]
    assert abs(front - chat * t) <= 2.5 / N
    behind = x < chat * t - 20.0 / N      # the second-order front spreads over ~15 cells here
    assert np.allclose(E[behind], 1.0, rtol=1e-4)
    assert np.all(out["Fx"][0, 0][behind] / E[behind] > 1 - 1e-6)
    # energy budget: everything in the box entered through the left face
    inside = E.sum() / N - 1e-10
    assert inside == pytest.approx(-st["boundary_E_out"], rel=1e-12)


# ----------------------------------------------------------------------------- P8 radiation wave

def _radwave_error(N, tau=0.1, eps=1e-6, theta=0.51, limiter="minmod"):
    chat = 1.0
    desc = wl.base_desc((N, 1, 1), (1.0 / N, 1.0, 1.0), bc="periodic", c=chat, exchange="absorb",
                        kappa_P=tau, kappa_F=tau, kappa_rho_pow=0, theta_F=theta, theta_E=theta,
                        limiter=limiter)
    x = (np.arange(N) + 0.5) / N
    E = 1.0 + eps * np.sin(2 * math.pi * x)
    shp = (1, 1, N)
    f = {"E": E.reshape(shp), "Fx": (chat * E).reshape(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
         "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None, "kP": None,
         "kF": None, "j": None}
    n = int(round(2.5 * N))
    dt = 1.0 / n          # = 0.4 dx / chat exactly; one wave period t_lambda = lambda / chat
    out, st = orc.subcycles({"desc": desc, "fields": f, "chat": chat, "dt": dt, "n_sub": n})
    assert st["n_realizability_fix"] == 0
    E1 = out["E"][0, 0]
    # perturbation only: the analytic wave eps e^{-chat k t} sin(2 pi (x - chat t)) after one period
    d_num = E1 - E1.mean()
    d_ex = eps * math.exp(-chat * tau * 1.0) * np.sin(2 * math.pi * x)
    return np.mean(np.abs(d_num - d_ex))


def test_radiation_wave_second_order():
    """Streaming radiation wave in an absorbing medium (Section 4.1.2): omega = chat k - i chat rho
    kappa, tau_lambda = 0.1, eps = 1e-6; the L1 error converges at second order."""
    p = GOLD["radwave_params"]["value"]
    errs = [_radwave_error(N, tau=p["tau_lambda"], eps=p["epsilon"]) for N in (32, 64, 128, 256)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert orders[-1] > 1.8 and orders[-2] > 1.7, (errs, orders)
    assert errs[-1] < 5e-3 * p["epsilon"]


def test_streaming_wave_second_order_with_mc_limiter():
    """The same wave without absorption (kappa = 0, so no splitting error floors the convergence):
    with the monotonized central limiter the L1 error converges at second order, and the wave's
    extrema are clipped less than by minmod (MC takes the central slope wherever neither difference
    exceeds three times the other).  Dropping MC's central argument (slope 2 min|d|, first order on
    smooth data) or its factor 2 (minmod) fails one of the two checks."""
    errs = [_radwave_error(N, tau=0.0, eps=1e-6, limiter="mc") for N in (32, 64, 128, 256)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders) > 1.9, (errs, orders)
    assert errs[-1] < 0.25 * _radwave_error(256, tau=0.0, eps=1e-6, limiter="minmod")


# ----------------------------------------------------------------------------- P9 dispersion

def _measure_omega(case, n_steps):
    cur = case
    out, _ = orc.subcycles(cur, n_sub=n_steps)
    x = (np.arange(case["desc"]["n"][0]) + 0.5) * case["desc"]["dx"][0]
    k = case["k"]
    a0 = np.mean((case["fields"]["E"][0, 0] - 1.0) * np.exp(-1j * k * x)) * 2
    a1 = np.mean((out["E"][0, 0] - 1.0) * np.exp(-1j * k * x)) * 2
    t = n_steps * case["dt"]
    return 1j * np.log(a1 / a0) / t


@pytest.mark.parametrize("tau,mode,theta,order,tol64", [
    (0.01, "equilibrium", 0.51, 1.8, 1e-3),
    (1.0, "equilibrium", 0.51, 0.8, 3e-3),
    (100.0, "equilibrium", 1.0, 1.8, 1e-2),
    (0.01, "frozen_t", 0.51, 1.8, 1e-3),
    (1.0, "frozen_t", 0.51, 0.8, 5e-3),
])
def test_linear_wave_dispersion(tau, mode, theta, order, tol64):
    """Linear radiation waves about E0 = 1, G0 = 0 with chi = 1/3: the Eddington mode travels at
    chat/sqrt(3) (Section 4.3.4) and, for radiative equilibrium, omega^2 + i chat kF omega -
    chat^2 k^2 / 3 = 0 (linearised Eqs. mixedframe:graysystem:radenergy/radmomentum); with a frozen
    emitting gas omega = +- chat k / sqrt(3) - i chat kF.  Unlimited slopes make the scheme linear.
    Where absorption and transport do not commute the operator split is first order in time
    (Section 3.1), so tau ~ 1 converges at first order; weak coupling converges at second order,
    and the stiff diffusion mode needs theta = 1 (Section 3.4)."""
    chat, k = 10.0, 2 * math.pi
    if mode == "frozen_t":
        w_ex = chat * k / math.sqrt(3.0) - 1j * chat * tau
        assert w_ex.real / (chat * k) == pytest.approx(GOLD["eddington_mode_speed"]["value"], rel=1e-15)
    else:
        disc = complex(-(chat * tau) ** 2 + 4 * chat ** 2 * k ** 2 / 3)
        roots = [(-1j * chat * tau + s * np.sqrt(disc)) / 2 for s in (1, -1)]
        w_ex = wl.dispersion_omega(chat, k, tau, mode)
        assert min(abs(w_ex - r) for r in roots) < 1e-12 * abs(w_ex)
    errs = []
    for N in (64, 128, 256):
        case = wl.config1(tau=tau, mode=mode, limiter="none", N=N, n_sub=0, theta=theta)
        n = int(round(0.05 / case["dt"]))
        w = _measure_omega(case, n)
        errs.append(abs(w - w_ex) / abs(w_ex))
    assert errs[0] < tol64, errs
    assert math.log2(errs[1] / errs[2]) > order, errs


# ----------------------------------------------------------------------------- P10 steady source

def test_steady_point_source_flux_falls_as_one_over_r():
    """Radiative equilibrium, gas at rest: in the steady state div F = j (no energy sink), so the
    flux through any circle enclosing the source is its luminosity L and |F| falls as 1/r in 2D
    (the concentrated-source problem of the abstract, with a transparent medium)."""
    N = 64
    case = wl.config2(N=N, n_sub=0)
    case["fields"]["kF"] = np.full_like(case["fields"]["kF"], 0.1)
    out, st = orc.subcycles(case, n_sub=int(round(3.0 / case["dt"])))
    assert st["n_nonfinite"] == 0
    X, Y, _ = wl.cell_centres(case["desc"], x0=(-1.0, -1.0, 0.0))
    r = np.sqrt(X ** 2 + Y ** 2)[0]
    Fr = ((out["Fx"] * X + out["Fy"] * Y) / np.where(r > 0, r, 1))[0]
    for r0 in (0.3, 0.45, 0.6, 0.75):
        ring = np.abs(r - r0) < 0.5 * case["desc"]["dx"][0]
        lum = Fr[ring].mean() * 2 * math.pi * r0
        assert lum == pytest.approx(case["L"], rel=0.05), (r0, lum)
    # flux-limiting condition everywhere (Eq. m1:fluxlimit)
    g = np.sqrt(out["Fx"] ** 2 + out["Fy"] ** 2) / case["desc"]["c"]
    assert np.all(g <= out["E"] * (1 + 1e-12))


# ----------------------------------------------------------------------------- P11 symmetries

def _smooth_case(n, seed, mode="equilibrium", beta_tau=False, limiter="minmod", closure="m1",
                 speeds="m1", kappa=1.0):
    case = wl.parity_case("sym", n, bc="periodic", exchange=mode, limiter=limiter, beta_tau=beta_tau,
                          closure=closure, speeds=speeds, kappa=kappa, n_sub=2, seed=seed)
    return case


def _permute(case, perm):
    """Relabel axes: new axis a is old axis perm[a] (arrays are (z, y, x))."""
    d = dict(case["desc"])
    d["n"] = tuple(case["desc"]["n"][perm[a]] for a in range(3))
    d["dx"] = tuple(case["desc"]["dx"][perm[a]] for a in range(3))
    f = case["fields"]
    # numpy axis of spatial dim a is 2 - a
    axes = [2 - perm[2 - ax] for ax in range(3)]
    names = ["Fx", "Fy", "Fz"]
    vnames = ["vx", "vy", "vz"]
    nf = {}
    for k, v in f.items():
        nf[k] = None if v is None else np.ascontiguousarray(np.transpose(v, axes))
    for a in range(3):
        nf[names[a]] = np.ascontiguousarray(np.transpose(f[names[perm[a]]], axes))
        src = f[vnames[perm[a]]]
        nf[vnames[a]] = None if src is None else np.ascontiguousarray(np.transpose(src, axes))
    return dict(case, desc=d, fields=nf), axes


@pytest.mark.parametrize("mode,beta_tau", [("equilibrium", False), ("full", True), ("absorb", False)])
def test_axis_permutation_symmetry(mode, beta_tau):
    case = _smooth_case((5, 6, 7), 21, mode=mode, beta_tau=beta_tau)
    out, _ = orc.subcycles(case)
    perm = (1, 2, 0)
    pc, axes = _permute(case, perm)
    pout, _ = orc.subcycles(pc)
    names = ["Fx", "Fy", "Fz"]
    for k in ("E", "T"):
        assert np.allclose(pout[k], np.transpose(out[k], axes), rtol=1e-13, atol=1e-14)
    for a in range(3):
        assert np.allclose(pout[names[a]], np.transpose(out[names[perm[a]]], axes), rtol=1e-13, atol=1e-13)


def test_mirror_symmetry():
    case = _smooth_case((6, 5, 4), 22, mode="full", beta_tau=True)
    out, _ = orc.subcycles(case)
    f = case["fields"]
    mf = {}
    for k, v in f.items():
        mf[k] = None if v is None else np.ascontiguousarray(v[:, :, ::-1])
    mf["Fx"] = -mf["Fx"]
    mf["vx"] = -mf["vx"]
    mout, _ = orc.subcycles(dict(case, fields=mf))
    assert np.allclose(mout["E"], out["E"][:, :, ::-1], rtol=1e-13, atol=0)
    assert np.allclose(mout["Fx"], -out["Fx"][:, :, ::-1], rtol=1e-13, atol=1e-13)
    assert np.allclose(mout["Fy"], out["Fy"][:, :, ::-1], rtol=1e-13, atol=1e-13)


def test_one_dimensional_embedding_is_bitwise():
    """A 3D grid whose data vary only along x gives exactly the 1D result (the transverse flux
    differences vanish identically)."""
    c1 = wl.parity_case("1d", (12, 1, 1), bc="periodic", exchange="full", beta_tau=True, n_sub=3, seed=5)
    o1, _ = orc.subcycles(c1)
    f3 = {}
    for k, v in c1["fields"].items():
        f3[k] = None if v is None else np.ascontiguousarray(np.broadcast_to(v, (3, 4, 12)))
    d3 = dict(c1["desc"], n=(12, 4, 3), dx=(c1["desc"]["dx"][0], 0.25, 1 / 3))
    o3, _ = orc.subcycles(dict(c1, desc=d3, fields=f3))
    for k in ("E", "Fx", "Fy", "Fz", "T"):
        assert np.array_equal(o3[k], np.broadcast_to(o1[k], (3, 4, 12))), k


def test_linearity_of_p1_fixed_speed_scheme():
    """With the P1 closure, fixed speeds -+chat/sqrt(3) and unlimited slopes, no sources, the
    subcycle is a linear map of U (the textbook HLL/Rusanov MUSCL-Hancock scheme for the
    telegraph system)."""
    g = np.random.default_rng(31)
    n = (8, 6, 5)
    desc = wl.base_desc(n, tuple(1.0 / v for v in n), bc="periodic", c=1.0, exchange="equilibrium",
                        limiter="none", closure="p1", speeds="fixed", kappa_P=0.0, kappa_F=0.0)
    shp = (n[2], n[1], n[0])
    X, Y, Z = wl.cell_centres(desc)

    def smooth():
        s = np.zeros(shp)
        for _ in range(4):
            kx, ky, kz = g.integers(-2, 3, size=3)
            s += g.normal() * np.cos(2 * math.pi * (kx * X + ky * Y + kz * Z) + g.uniform(0, 6.3))
        return s

    def state():
        return {"E": 4.0 + 0.2 * smooth(), "Fx": 0.2 * smooth(), "Fy": 0.2 * smooth(), "Fz": 0.2 * smooth(),
                "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None, "kP": None,
                "kF": None, "j": None}

    u1, u2 = state(), state()
    a, b = 0.3, 0.7
    u3 = dict(u1)
    for k in ("E", "Fx", "Fy", "Fz"):
        u3[k] = a * u1[k] + b * u2[k]
    base = {"desc": desc, "chat": 1.0, "dt": wl.cfl_dt(desc, 1.0), "n_sub": 3}
    o1, s1 = orc.subcycles(dict(base, fields=u1))
    o2, _ = orc.subcycles(dict(base, fields=u2))
    o3, _ = orc.subcycles(dict(base, fields=u3))
    assert s1["n_face_fallback"] == 0
    for k in ("E", "Fx", "Fy", "Fz"):
        assert np.allclose(o3[k], a * o1[k] + b * o2[k], rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------- P12 brute force

def _py_subcycle(case):
    """Independent straight-line re-evaluation of one subcycle in Python floats, written from the
    paper's formulas and the same readings (small grids only)."""
    d = case["desc"]
    n = d["n"]
    c, chat, dt = d["c"], case["chat"], case["dt"]
    act = [n[a] > 1 for a in range(3)]
    f = case["fields"]

    def bc_map(idx, allow_dir):
        idx = list(idx)
        sg = [1.0, 1.0, 1.0]
        for a in range(3):
            while idx[a] < 0 or idx[a] >= n[a]:
                low = idx[a] < 0
                bc = d["bc_lo"][a] if low else d["bc_hi"][a]
                if bc == "dirichlet" and allow_dir:
                    return None, (a, low), sg
                if bc == "periodic":
                    idx[a] %= n[a]
                elif bc in ("outflow", "dirichlet"):
                    idx[a] = 0 if low else n[a] - 1
                else:
                    idx[a] = -idx[a] - 1 if low else 2 * n[a] - 1 - idx[a]
                    sg[a] = -sg[a]
        return idx, None, sg

    def U_m(i, j, k):
        idx, dirf, sg = bc_map((i, j, k), True)
        if idx is None:
            a, low = dirf
            s = d["dirichlet_lo"][a] if low else d["dirichlet_hi"][a]
            return [s[0], s[1] / c, s[2] / c, s[3] / c]
        x, y, z = idx
        return [f["E"][z, y, x], sg[0] * (f["Fx"][z, y, x] / c), sg[1] * (f["Fy"][z, y, x] / c),
                sg[2] * (f["Fz"][z, y, x] / c)]

    def gas(i, j, k):
        idx, _, sg = bc_map((i, j, k), False)
        x, y, z = idx
        rho = f["rho"][z, y, x]
        v = [0.0 if f[nm] is None else sg[a] * f[nm][z, y, x] for a, nm in enumerate(("vx", "vy", "vz"))]
        pw = d["kappa_rho_pow"]
        law = lambda kap: kap if pw == 0 else (kap * rho if pw == 1 else (kap * rho) * rho)
        kP = law(d["kappa_P"]) if f["kP"] is None else f["kP"][z, y, x]
        kF = law(d["kappa_F"]) if f["kF"] is None else f["kF"][z, y, x]
        jj = 0.0 if f["j"] is None else f["j"][z, y, x]
        return rho, f["T"][z, y, x], v, kP, kF, jj

    def flux(U, a):
        E, G = U[0], U[1:]
        g = math.sqrt(G[0] ** 2 + G[1] ** 2 + G[2] ** 2)
        ff = min(g / E, 1.0)
        chi = (3 + 4 * ff * ff) / (5 + 2 * math.sqrt(4 - 3 * ff * ff))
        nv = [G[b] / g for b in range(3)] if g > 0 else [0.0, 0.0, 0.0]
        T = [[(1 - chi) / 2 * (b == e) + (3 * chi - 1) / 2 * nv[b] * nv[e] for e in range(3)] for b in range(3)]
        mu = nv[a]
        s = math.sqrt(4 - 3 * ff * ff)
        rad = max(0.0, (2 / 3) * (4 - 3 * ff * ff - s) + 2 * mu * mu * (2 - ff * ff - s))
        return ([chat * G[a]] + [chat * E * T[a][e] for e in range(3)],
                chat * (mu * ff - math.sqrt(rad)) / s, chat * (mu * ff + math.sqrt(rad)) / s)

    def hll(UL, UR, a):
        FL, l1L, l3L = flux(UL, a)
        FR, l1R, l3R = flux(UR, a)
        SRp, SLm = max(max(l3L, l3R), 0.0), min(min(l1L, l1R), 0.0)
        if SRp - SLm <= 0:
            return [0.5 * (FL[q] + FR[q]) for q in range(4)]
        return [(SRp * FL[q] - SLm * FR[q] + SRp * SLm * (UR[q] - UL[q])) / (SRp - SLm) for q in range(4)]

    def explicit(U, g_):
        rho, T, v, kP, kF, jj = g_
        S = [chat * jj / c, 0.0, 0.0, 0.0]
        if d["beta_tau"]:
            S[0] += chat * kF * sum((v[a] / c) * U[1 + a] for a in range(3))
            for a in range(3):
                S[1 + a] += chat * (4 / 3) * kF * U[0] * (v[a] / c)
        return S

    def theta_fac(th, x):
        return (1 - (1 - th) * x) / (1 + th * x)

    def direct(U, g_, h):
        rho, T, v, kP, kF, jj = g_
        fF = theta_fac(d["theta_F"], chat * kF * h)
        U = [U[0], U[1] * fF, U[2] * fF, U[3] * fF]
        if d["exchange"] == "absorb":
            U[0] *= theta_fac(d["theta_E"], chat * kP * h)
        elif d["exchange"] == "frozen_t":
            x = chat * kP * h
            U[0] = (U[0] * (1 - (1 - d["theta_E"]) * x) + x * d["a_rad"] * T ** 4) / (1 + d["theta_E"] * x)
        return U

    def realize(U):
        U = list(U)
        U[0] = max(U[0], d["E_floor"])
        g2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
        if g2 > U[0] ** 2:
            s = U[0] / math.sqrt(g2)
            U[1:] = [u * s for u in U[1:]]
        return U

    E_ = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    rng_ = [range(-2 if act[a] else 0, n[a] + (2 if act[a] else 0)) for a in range(3)]
    Uh = {}
    for k in rng_[2]:
        for j in rng_[1]:
            for i in rng_[0]:
                U0 = U_m(i, j, k)
                div = [0.0] * 4
                for a in range(3):
                    if not act[a]:
                        continue
                    e = E_[a]
                    Fl = hll(U_m(i - e[0], j - e[1], k - e[2]), U0, a)
                    Fr = hll(U0, U_m(i + e[0], j + e[1], k + e[2]), a)
                    div = [div[q] + (Fr[q] - Fl[q]) / d["dx"][a] for q in range(4)]
                g_ = gas(i, j, k)
                S = explicit(U0, g_)
                U = [U0[q] - 0.5 * dt * div[q] + 0.5 * dt * S[q] for q in range(4)]
                Uh[(i, j, k)] = realize(direct(U, g_, 0.5 * dt))

    def slope(i, j, k, a):
        e = E_[a]
        um, u0, up = Uh[(i - e[0], j - e[1], k - e[2])], Uh[(i, j, k)], Uh[(i + e[0], j + e[1], k + e[2])]
        s = []
        for q in range(4):
            dl, dr = u0[q] - um[q], up[q] - u0[q]
            if d["limiter"] == "none":
                s.append(0.5 * (dl + dr))
            elif dl * dr <= 0:
                s.append(0.0)
            elif d["limiter"] == "minmod":
                s.append(math.copysign(min(abs(dl), abs(dr)), dl))
            else:
                s.append(math.copysign(min(2 * min(abs(dl), abs(dr)), 0.5 * abs(dl + dr)), dl))
        for sgn in (-1, 1):
            fu = [u0[q] + sgn * 0.5 * s[q] for q in range(4)]
            if not fu[0] > 0 or fu[1] ** 2 + fu[2] ** 2 + fu[3] ** 2 > (1 + 1e-12) * fu[0] ** 2:
                return [0.0] * 4
        return s

    out = {k: np.zeros_like(f["E"]) for k in ("E", "Fx", "Fy", "Fz", "T")}
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                div = [0.0] * 4
                for a in range(3):
                    if not act[a]:
                        continue
                    e = E_[a]
                    cm = (i - e[0], j - e[1], k - e[2])
                    cp = (i + e[0], j + e[1], k + e[2])
                    s_m, s_0, s_p = slope(*cm, a), slope(i, j, k, a), slope(*cp, a)
                    UL_l = [Uh[cm][q] + 0.5 * s_m[q] for q in range(4)]
                    UR_l = [Uh[(i, j, k)][q] - 0.5 * s_0[q] for q in range(4)]
                    UL_r = [Uh[(i, j, k)][q] + 0.5 * s_0[q] for q in range(4)]
                    UR_r = [Uh[cp][q] - 0.5 * s_p[q] for q in range(4)]
                    Fl = hll(UL_l, UR_l, a)
                    Fr = hll(UL_r, UR_r, a)
                    div = [div[q] + (Fr[q] - Fl[q]) / d["dx"][a] for q in range(4)]
                g_ = gas(i, j, k)
                S = explicit(Uh[(i, j, k)], g_)
                U0 = U_m(i, j, k)
                U = direct([U0[q] - dt * div[q] + dt * S[q] for q in range(4)], g_, dt)
                T = g_[1]
                if d["exchange"] == "full":
                    U[0] = max(U[0], d["E_floor"])
                    e1, T1, _ = orc.exchange_full(d, chat, dt, g_[0], g_[3], U[0], T)
                    U[0], T = e1, T1
                U = realize(U)
                out["E"][k, j, i] = U[0]
                out["Fx"][k, j, i] = c * U[1]
                out["Fy"][k, j, i] = c * U[2]
                out["Fz"][k, j, i] = c * U[3]
                out["T"][k, j, i] = T
    return out


BRUTE_CASES = [
    dict(n=(3, 4, 3), bc="periodic", exchange="full", beta_tau=True, limiter="minmod", with_j=True),
    dict(n=(4, 3, 1), bc="outflow", exchange="absorb", limiter="mc"),
    dict(n=(5, 3, 3), bc="reflect", exchange="frozen_t", limiter="minmod", beta_tau=True),
    dict(n=(6, 1, 1), bc="periodic", exchange="equilibrium", limiter="none", kP_array=True),
    dict(n=(4, 4, 1), bc=(["dirichlet", "outflow", "periodic"], ["reflect", "dirichlet", "periodic"]),
         exchange="equilibrium", limiter="minmod",
         dirichlet=([[1.0, 0.5, 0.1, 0.0], [0.8, 0.0, -0.3, 0.0], [0.0] * 4],
                    [[0.0] * 4, [1.2, 0.2, 0.4, 0.0], [0.0] * 4])),
]


@pytest.mark.parametrize("idx", range(len(BRUTE_CASES)))
def test_brute_force_reevaluation(idx):
    kw = dict(BRUTE_CASES[idx])
    n = kw.pop("n")
    case = wl.parity_case(f"brute{idx}", n, n_sub=1, seed=40 + idx, fmax=0.95, **kw)
    ref = _py_subcycle(case)
    out, _ = orc.subcycles(case)
    for k in ("E", "Fx", "Fy", "Fz"):
        scale = np.max(np.abs(ref["E"])) * (case["desc"]["c"] if k != "E" else 1.0)
        assert np.max(np.abs(out[k] - ref[k])) <= 1e-14 * scale, k
    if case["desc"]["exchange"] == "full":
        assert np.allclose(out["T"], ref["T"], rtol=1e-14, atol=0)


def test_long_run_stays_finite_and_realizable():
    case = wl.parity_case("long", (6, 6, 6), bc="periodic", exchange="full", beta_tau=True, n_sub=300,
                          seed=50, with_j=True, kappa=5.0)
    out, st = orc.subcycles(case)
    assert st["n_nonfinite"] == 0
    g = np.sqrt(out["Fx"] ** 2 + out["Fy"] ** 2 + out["Fz"] ** 2) / case["desc"]["c"]
    assert np.all(g <= out["E"] * (1 + 1e-14)) and np.all(out["E"] > 0) and np.all(out["T"] > 0)
