"""Seeded synthetic inputs for the radiation subcycle (initial and frozen-gas states only).

This module holds no step of the method: it only draws and shapes input fields.  Both the
CUDA path (through the C-ABI binding) and the CPU oracle consume the plain dicts it returns:

    case = {"name": str, "desc": {...grid and physics parameters...},
            "fields": {"E", "Fx", "Fy", "Fz", "T", "rho", "vx", "vy", "vz", "kP", "kF", "j"},
            "chat": float, "dt": float, "n_sub": int}

Arrays are float64, C-ordered with shape (nz, ny, nx) (x fastest).  Absent optional fields are
None (zero velocity, the opacity law k = kappa * rho^p, no emissivity).  Units: a_R = 1 and
k_B/mu = 1 unless stated, so P = rho T and e = rho T / (gamma - 1).

The workloads mirror the paper's radiation-subsystem tests (Section 4.1), its concentrated-source
problem (abstract; Eq. radshell:sourceprofile) and its dusty-shell problem (Section 4.3.6); the
paper uses no external datasets.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 13060010


def rng(offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + offset))


def base_desc(n, dx, bc="periodic", **kw):
    d = {
        "n": tuple(int(v) for v in n),
        "dx": tuple(float(v) for v in dx),
        "bc_lo": [bc] * 3 if isinstance(bc, str) else list(bc[0]),
        "bc_hi": [bc] * 3 if isinstance(bc, str) else list(bc[1]),
        "dirichlet_lo": [[0.0] * 4 for _ in range(3)],
        "dirichlet_hi": [[0.0] * 4 for _ in range(3)],
        "c": 1.0,
        "a_rad": 1.0,
        "gamma": 5.0 / 3.0,
        "mu_over_kB": 1.0,
        "theta_F": 1.0,
        "theta_E": 1.0,
        "E_floor": 1e-30,
        "exchange": "equilibrium",
        "beta_tau": False,
        "limiter": "minmod",
        "closure": "m1",
        "speeds": "m1",
        "kappa_P": 0.0,
        "kappa_F": 0.0,
        "kappa_rho_pow": 0,
        "cfl": 0.4,
        "precision": "fp64",
        "linear_eps": 1.0,
    }
    d.update(kw)
    return d


def cfl_dt(desc, chat, cfl=None):
    cfl = desc.get("cfl", 0.4) if cfl is None else cfl
    dxs = [desc["dx"][d] for d in range(3) if desc["n"][d] > 1]
    return cfl * min(dxs) / chat if dxs else cfl / chat


def _shape(desc):
    nx, ny, nz = desc["n"]
    return (nz, ny, nx)


def cell_centres(desc, x0=(0.0, 0.0, 0.0)):
    nx, ny, nz = desc["n"]
    dx = desc["dx"]
    x = x0[0] + (np.arange(nx) + 0.5) * dx[0]
    y = x0[1] + (np.arange(ny) + 0.5) * dx[1]
    z = x0[2] + (np.arange(nz) + 0.5) * dx[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def random_directions(g: np.random.Generator, shape):
    """Unit vectors uniform on the sphere."""
    z = g.uniform(-1.0, 1.0, size=shape)
    phi = g.uniform(0.0, 2.0 * math.pi, size=shape)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return r * np.cos(phi), r * np.sin(phi), z


def random_state(desc, g: np.random.Generator, fmax=0.9, Emin=0.5, Emax=2.0, dims_active=None):
    """Random realizable radiation state: E uniform in [Emin, Emax], F = c E f n with f uniform
    in [0, fmax] and n uniform on the sphere (restricted to the active directions)."""
    shp = _shape(desc)
    E = g.uniform(Emin, Emax, size=shp)
    f = g.uniform(0.0, fmax, size=shp)
    nx, ny, nz = random_directions(g, shp)
    act = [desc["n"][d] > 1 for d in range(3)] if dims_active is None else dims_active
    comps = [nx, ny, nz]
    for d in range(3):
        if not act[d]:
            comps[d] = np.zeros(shp)
    norm = np.sqrt(comps[0] ** 2 + comps[1] ** 2 + comps[2] ** 2)
    norm = np.where(norm > 0, norm, 1.0)
    c = desc["c"]
    return {
        "E": E,
        "Fx": c * E * f * comps[0] / norm,
        "Fy": c * E * f * comps[1] / norm,
        "Fz": c * E * f * comps[2] / norm,
    }


# ----------------------------------------------------------------------------- small parity cases

def parity_case(name, n, bc="periodic", exchange="equilibrium", limiter="minmod", beta_tau=False,
                closure="m1", speeds="m1", kappa=1.0, kappa_rho_pow=1, theta=1.0, chat=1.0, c=10.0,
                n_sub=3, seed=0, with_j=False, with_v=None, fmax=0.9, dirichlet=None,
                precision="fp64", kP_array=False, dx=None):
    """Random realizable radiation state on a small grid with a random frozen gas state."""
    g = rng(1000 + seed)
    n = tuple(n)
    if dx is None:
        dx = tuple(1.0 / max(v, 1) for v in n)
    desc = base_desc(n, dx, bc=bc, c=c, exchange=exchange, limiter=limiter, beta_tau=beta_tau,
                     closure=closure, speeds=speeds, kappa_P=kappa, kappa_F=kappa,
                     kappa_rho_pow=kappa_rho_pow, theta_F=theta, theta_E=theta, E_floor=1e-12,
                     precision=precision)
    if dirichlet is not None:
        desc["dirichlet_lo"], desc["dirichlet_hi"] = dirichlet
    shp = _shape(desc)
    st = random_state(desc, g, fmax=fmax)
    rho = np.exp(g.normal(0.0, 0.5, size=shp))
    T = np.exp(g.normal(0.0, 0.2, size=shp))
    if exchange == "full":
        # start near radiative equilibrium so the coupled problem is not violently stiff
        st["E"] = desc["a_rad"] * T ** 4 * g.uniform(0.7, 1.3, size=shp)
        f = g.uniform(0.0, fmax, size=shp)
        nx_, ny_, nz_ = random_directions(g, shp)
        act = [n[d] > 1 for d in range(3)]
        comps = [nx_ if act[0] else 0 * nx_, ny_ if act[1] else 0 * ny_, nz_ if act[2] else 0 * nz_]
        norm = np.sqrt(sum(cc ** 2 for cc in comps))
        norm = np.where(norm > 0, norm, 1.0)
        for d, k in enumerate(("Fx", "Fy", "Fz")):
            st[k] = c * st["E"] * f * comps[d] / norm
    v = with_v if with_v is not None else beta_tau
    fields = dict(st)
    fields["T"] = T
    fields["rho"] = rho
    if v:
        for k in ("vx", "vy", "vz"):
            fields[k] = g.normal(0.0, 0.05 * c, size=shp)
    else:
        fields["vx"] = fields["vy"] = fields["vz"] = None
    fields["kP"] = fields["kF"] = None
    if kP_array:
        fields["kP"] = kappa * rho * g.uniform(0.5, 1.5, size=shp)
        fields["kF"] = kappa * rho * g.uniform(0.5, 1.5, size=shp)
    fields["j"] = g.uniform(0.0, 2.0, size=shp) if with_j else None
    dt = cfl_dt(desc, chat)
    return {"name": name, "desc": desc, "fields": fields, "chat": chat, "dt": dt, "n_sub": n_sub}


def stiff_case(name, n, uniform=False, exchange="full", K=2.0e4, x_abs=20.0, rho0=1000.0, T0=1.5, theta=1.0,
               c=10.0, chat=1.0, n_sub=10, seed=0, bc="periodic", fmax=0.5, precision="split"):
    """Stiff exchange with the gas energy far above the radiation's: hot dense gas against a weak
    radiation field.  K = e / ((c/chat) E) sets E from the gas (e = rho T / ((gamma - 1) mu/k_B)), and
    the opacity law k = kappa rho (kappa_P = kappa_F) gives chat k dt = x_abs at rho0.  The density is
    rounded to FP32 (so the split path's FP32 copy of it is exact) and v = 0, j = 0 (no explicit
    source).  uniform: every cell holds the same state, so the transport of every subcycle cancels
    exactly and only the stiff sources act; otherwise rho = rho0 exp(N(0, 0.3^2)), T = T0 exp(N(0,
    0.1^2)), E = E_K U(0.5, 1.5) and F = c E f n with f ~ U(0, fmax), n uniform on the sphere (active
    directions only)."""
    g = rng(5000 + seed)
    n = tuple(n)
    dx = tuple(1.0 / max(v, 1) for v in n)
    desc = base_desc(n, dx, bc=bc, c=c, exchange=exchange, kappa_rho_pow=1, theta_F=theta, theta_E=theta,
                     E_floor=1e-12, precision=precision)
    dt = cfl_dt(desc, chat)
    kappa = float(np.float32(x_abs / (chat * rho0 * dt)))
    desc["kappa_P"] = desc["kappa_F"] = kappa
    shp = _shape(desc)
    gm1_mu = (desc["gamma"] - 1.0) * desc["mu_over_kB"]
    if uniform:
        rho = np.full(shp, float(np.float32(rho0)))
        T = np.full(shp, T0)
        E = np.full(shp, rho0 * T0 / gm1_mu / (K * c / chat))
        f = np.full(shp, 0.5 * fmax)
        dirs = [np.full(shp, v) for v in (0.48, -0.6, 0.64)]
    else:
        rho = (rho0 * np.exp(g.normal(0.0, 0.3, size=shp))).astype(np.float32).astype(np.float64)
        T = T0 * np.exp(g.normal(0.0, 0.1, size=shp))
        E = rho0 * T0 / gm1_mu / (K * c / chat) * g.uniform(0.5, 1.5, size=shp)
        f = g.uniform(0.0, fmax, size=shp)
        dirs = list(random_directions(g, shp))
    act = [n[d] > 1 for d in range(3)]
    comps = [dirs[d] if act[d] else np.zeros(shp) for d in range(3)]
    norm = np.sqrt(sum(cc ** 2 for cc in comps))
    norm = np.where(norm > 0, norm, 1.0)
    fields = {"E": E, "T": T, "rho": rho, "vx": None, "vy": None, "vz": None, "kP": None, "kF": None, "j": None}
    for d, k in enumerate(("Fx", "Fy", "Fz")):
        fields[k] = c * E * f * comps[d] / norm
    return {"name": name, "desc": desc, "fields": fields, "chat": chat, "dt": dt, "n_sub": n_sub}


# cgs constants of the physical-units cases
A_RAD_CGS = 7.5657e-15        # erg cm^-3 K^-4
C_CGS = 2.99792458e10         # cm s^-1
MU_OVER_KB_CGS = 0.6 * 1.6726e-24 / 1.380649e-16  # mean mass per particle over k_B (mu = 0.6), g K erg^-1

# (density g cm^-3, gas temperature K, cell size cm, opacity cm^2 g^-1, c / chat, velocity dispersion cm s^-1)
PHYSICAL_REGIMES = {
    "protostellar_disk": (1e-10, 300.0, 1.496e13 / 8, 1.0, 100.0, 1e5),
    "stellar_envelope": (1e-7, 1e5, 7e9, 0.4, 30.0, 1e6),
    "molecular_cloud": (1e-22, 20.0, 3.086e17, 10.0, 1000.0, 1e5),
}


def physical_units_case(name, n, regime, precision="split", n_sub=4, seed=0, fmax=0.6):
    """A state in cgs units (a_R, c and mu/k_B of an ionised gas with mu = 0.6), for the ranges of the
    split path's FP32 arithmetic: rho = rho0 exp(N(0, 0.5^2)), T = T0 exp(N(0, 0.2^2)), radiation
    temperature T U(0.6, 1.3) (E = a_R T_rad^4), F = c E f n with f ~ U(0, fmax), v ~ N(0, sigma_v^2) per
    component, the opacity law k = kappa rho, FULL exchange with beta tau terms, chat = c / (c / chat)
    and dt at CFL 0.4.  Density and velocity are rounded to FP32 (the split path's copies of them are
    then exact).  The regimes span optically thick and stiff (disk: chat k dt ~ 75; stellar envelope ~
    110) to optically thin (molecular cloud, chat k dt ~ 1e-4), with E from 1e-9 to 1e6 erg cm^-3."""
    rho0, T0, dx0, kappa, c_over_chat, sig_v = PHYSICAL_REGIMES[regime]
    g = rng(7000 + seed)
    n = tuple(n)
    dx = tuple(dx0 for _ in n)
    desc = base_desc(n, dx, c=C_CGS, a_rad=A_RAD_CGS, mu_over_kB=MU_OVER_KB_CGS, exchange="full",
                     beta_tau=True, kappa_P=kappa, kappa_F=kappa, kappa_rho_pow=1, E_floor=1e-30,
                     precision=precision)
    chat = C_CGS / c_over_chat
    shp = _shape(desc)
    rho = (rho0 * np.exp(g.normal(0.0, 0.5, size=shp))).astype(np.float32).astype(np.float64)
    T = T0 * np.exp(g.normal(0.0, 0.2, size=shp))
    E = A_RAD_CGS * (T * g.uniform(0.6, 1.3, size=shp)) ** 4
    f = g.uniform(0.0, fmax, size=shp)
    dirs = list(random_directions(g, shp))
    act = [n[d] > 1 for d in range(3)]
    comps = [dirs[d] if act[d] else np.zeros(shp) for d in range(3)]
    norm = np.sqrt(sum(cc ** 2 for cc in comps))
    norm = np.where(norm > 0, norm, 1.0)
    fields = {"E": E, "T": T, "rho": rho, "kP": None, "kF": None, "j": None}
    for d, k in enumerate(("Fx", "Fy", "Fz")):
        fields[k] = C_CGS * E * f * comps[d] / norm
    for k in ("vx", "vy", "vz"):
        fields[k] = g.normal(0.0, sig_v, size=shp).astype(np.float32).astype(np.float64)
    return {"name": name, "desc": desc, "fields": fields, "chat": chat, "dt": cfl_dt(desc, chat), "n_sub": n_sub}


def gas_case(name, n, bc="periodic", limiter="minmod", beta_tau=True, kappa=2.0, kappa_rho_pow=1, kF_array=False,
             seed=0, precision="fp64", dirichlet=None, exchange="full", n_sub=4, with_v=True, c=10.0, gamma=5.0 / 3.0):
    """A gas-step case: the random gas and radiation of parity_case (rho = exp(N(0, 0.5^2)), T = exp(N(0,
    0.2^2)), v ~ N(0, (0.05 c)^2) per component, Mach numbers up to about 1), a second random radiation
    state "rad1" (the radiation at t^{n+1} for the source correction), dt_gas = 0.1 min(dx) (below a
    third of the gas Courant limit) and n_sub radiation subcycles of dt_gas / n_sub."""
    case = parity_case(name, n, bc=bc, exchange=exchange, limiter=limiter, beta_tau=beta_tau, kappa=kappa,
                       kappa_rho_pow=kappa_rho_pow, seed=seed, with_v=with_v, precision=precision,
                       dirichlet=dirichlet, kP_array=kF_array, c=c, n_sub=n_sub)
    case["desc"]["gamma"] = gamma
    g = rng(3000 + seed)
    case["rad1"] = random_state(case["desc"], g, fmax=0.9)
    dxs = [case["desc"]["dx"][d] for d in range(3) if case["desc"]["n"][d] > 1]
    case["dt_gas"] = 0.1 * min(dxs)
    case["dt"] = case["dt_gas"] / n_sub
    return case


def radpulse_case(N=512, v=3e6, shift=None, beta_tau=True):
    """The advected radiation pulse (Section 4.3.2) in cgs units: rho_0 = 25 g cm^-3, T_0 = 1.1e7 K,
    w = 20 cm, mu = m_H, kappa_0 = 0.4 cm^2 g^-1, gamma = 5/3, periodic x / w in [-21.25, 21.25] on N cells;
    T / T_0 = 1 + exp(-x^2 / (2 w^2)) about x = -shift (default: v t_end = 2 w for a moving run, 0 at rest),
    rho from pressure equilibrium (Eq. radpulse:rho), E = a_R T^4, F the quasi-steady flux
    -c dE/dx / (3 rho kappa_0) + (4/3) v E (reading), uniform velocity v; chat = 100 a_0; M1 closure, MC
    limiter, FULL exchange, theta = 1.  Also returns t_end = 2 w / 3e6 cm s^-1."""
    kB, mH, aR, c = 1.380649e-16, 1.6726e-24, 7.5657e-15, 2.99792458e10
    rho0, T0, w, kap, gam = 25.0, 1.1e7, 20.0, 0.4, 5.0 / 3.0
    t_end = 2.0 * w / 3e6
    if shift is None:
        shift = v * t_end
    mu = mH / kB
    a0 = math.sqrt(gam * T0 / mu)
    P0 = aR * T0 ** 4 / (rho0 * a0 ** 2)
    L = 42.5 * w
    dx = L / N
    x = -0.5 * L + (np.arange(N) + 0.5) * dx
    xs = (x + shift + 0.5 * L) % L - 0.5 * L
    T = T0 * (1.0 + np.exp(-xs ** 2 / (2 * w * w)))
    rho = rho0 * (T0 / T + gam * P0 / 3.0 * (T0 / T - (T / T0) ** 3))
    E = aR * T ** 4
    dEdx = (np.roll(E, -1) - np.roll(E, 1)) / (2 * dx)
    F = -c / (3 * rho * kap) * dEdx + (4.0 / 3.0) * v * E
    desc = base_desc((N, 1, 1), (dx, 1.0, 1.0), bc="periodic", c=c, a_rad=aR, gamma=gam, mu_over_kB=mu,
                     exchange="full", beta_tau=beta_tau, limiter="mc", kappa_P=kap, kappa_F=kap, kappa_rho_pow=1,
                     theta_F=1.0, theta_E=1.0, E_floor=1e-30, cfl=0.4)
    sh = (1, 1, N)
    z = np.zeros(sh)
    fields = {"E": E.reshape(sh), "Fx": F.reshape(sh), "Fy": z, "Fz": z.copy(), "T": T.reshape(sh),
              "rho": rho.reshape(sh), "vx": np.full(sh, float(v)), "vy": z.copy(), "vz": z.copy(), "kP": None,
              "kF": None, "j": None}
    return {"name": f"radpulse{N}", "desc": desc, "fields": fields, "chat": 100.0 * a0, "t_end": t_end, "P0": P0}


# ----------------------------------------------------------------------------- paper-shaped configs

def dispersion_omega(chat, k, kF, mode):
    """Continuum frequency of the linear radiation mode about (E0, G0 = 0) with chi = 1/3 (used only
    to set up the eigenmode initial state; see Eqs. mixedframe:graysystem:radenergy/radmomentum)."""
    if mode == "frozen_t":
        return chat * k / math.sqrt(3.0) - 1j * chat * kF
    disc = complex(-(chat * kF) ** 2 + 4.0 * chat ** 2 * k ** 2 / 3.0)
    r = np.sqrt(disc)
    w1 = (-1j * chat * kF + r) / 2.0
    w2 = (-1j * chat * kF - r) / 2.0
    # propagating branch with positive phase speed, else the slowly damped diffusion mode
    if abs(w1.real) > 1e-14 * abs(w1):
        return w1 if w1.real > 0 else w2
    return w1 if abs(w1.imag) < abs(w2.imag) else w2


def config1(tau=1.0, mode="equilibrium", limiter="minmod", N=512, n_sub=1000, eps=1e-6, theta=0.51,
            chat=10.0):
    """1D radiation-only linear wave: N periodic cells on [0, 1), static uniform gas (rho = 1, T = 1,
    v = 0), E0 = 1, F0 = 0, dE = eps cos(2 pi x), F on the eigenmode, uniform absorption with optical
    depth tau per wavelength, chat = c = 10, CFL 0.4."""
    dx = 1.0 / N
    desc = base_desc((N, 1, 1), (dx, 1.0, 1.0), bc="periodic", c=chat, exchange=mode, limiter=limiter,
                     kappa_P=tau, kappa_F=tau, kappa_rho_pow=0, theta_F=theta, theta_E=theta,
                     E_floor=1e-30)
    x = (np.arange(N) + 0.5) * dx
    k = 2.0 * math.pi
    w = dispersion_omega(chat, k, tau, mode)
    dE = eps * np.exp(1j * k * x)
    E = 1.0 + dE.real
    # eigenvector of the linearised radiation-energy equation: -i w dE + i chat k dG = -chat kP dE
    # (the right-hand side is present only with an emitting gas at fixed temperature)
    kP_eff = tau if mode == "frozen_t" else 0.0
    G = (((w + 1j * chat * kP_eff) / (chat * k)) * dE).real
    shp = (1, 1, N)
    fields = {
        "E": E.reshape(shp), "Fx": (desc["c"] * G).reshape(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
        "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None,
        "kP": None, "kF": None, "j": None,
    }
    return {"name": f"config1_tau{tau}_{mode}", "desc": desc, "fields": fields, "chat": chat,
            "dt": cfl_dt(desc, chat), "n_sub": n_sub, "omega": w, "k": k}


def config2(N=256, n_sub=2000, L=1.0, sigma=0.05):
    """2D concentrated source: N x N on [-1, 1]^2, outflow, static gas, Gaussian emissivity of width
    sigma (2D normalisation) at the centre, kF = 1000 for r < 0.1 and 0.1 outside, chat = c = 1."""
    dx = 2.0 / N
    desc = base_desc((N, N, 1), (dx, dx, 1.0), bc="outflow", c=1.0, exchange="equilibrium",
                     kappa_P=0.0, kappa_F=0.0, theta_F=1.0, theta_E=1.0, E_floor=1e-10)
    X, Y, _ = cell_centres(desc, x0=(-1.0, -1.0, 0.0))
    r2 = X ** 2 + Y ** 2
    j = L * np.exp(-r2 / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2)
    kF = np.where(r2 < 0.1 ** 2, 1000.0, 0.1)
    shp = X.shape
    fields = {
        "E": np.full(shp, 1e-10), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
        "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None,
        "kP": np.zeros(shp), "kF": kF, "j": j,
    }
    return {"name": "config2_source2d", "desc": desc, "fields": fields, "chat": 1.0,
            "dt": cfl_dt(desc, 1.0), "n_sub": n_sub, "L": L, "sigma": sigma}


def config3(N=256, n_sub=25, precision="split"):
    """3D dusty shell: [-0.5, 0.5]^3, outflow, rho = 1 ambient and 100 in the shell 0.3 <= r <= 0.35,
    uniform kappa with shell optical depth 10 (k = 2 rho), Gaussian point luminosity L = 1 of width
    2 dx, FULL exchange at T0 = 1 with E = a_R T0^4, O(beta tau) terms on, theta = 1, radial
    expansion 1 (about the sound speed) inside the shell, chat = 50 v_max, c = 10 chat."""
    dx = 1.0 / N
    gamma = 5.0 / 3.0
    cs = math.sqrt(gamma)
    vmax = 1.0 + cs
    chat = 50.0 * vmax
    c = 10.0 * chat
    desc = base_desc((N, N, N), (dx, dx, dx), bc="outflow", c=c, gamma=gamma, exchange="full",
                     beta_tau=True, kappa_P=2.0, kappa_F=2.0, kappa_rho_pow=1, theta_F=1.0, theta_E=1.0,
                     E_floor=1e-20, precision=precision)
    X, Y, Z = cell_centres(desc, x0=(-0.5, -0.5, -0.5))
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    shell = (r >= 0.3) & (r <= 0.35)
    rho = np.where(shell, 100.0, 1.0)
    sig = 2.0 * dx
    j = np.exp(-r ** 2 / (2 * sig ** 2)) / (2 * math.pi * sig ** 2) ** 1.5
    rs = np.where(r > 0, r, 1.0)
    vr = np.where(shell, 1.0, 0.0)
    shp = X.shape
    fields = {
        "E": np.ones(shp), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
        "T": np.ones(shp), "rho": rho, "vx": vr * X / rs, "vy": vr * Y / rs, "vz": vr * Z / rs,
        "kP": None, "kF": None, "j": j,
    }
    return {"name": f"config3_shell{N}", "desc": desc, "fields": fields, "chat": chat,
            "dt": cfl_dt(desc, chat), "n_sub": n_sub}


def lognormal_field(N, g: np.random.Generator, sigma=1.0, slope=-11.0 / 3.0):
    """ln rho: Gaussian random field with power spectrum P(k) ~ k^slope, unit variance scaled to
    sigma, mean -sigma^2/2 (so <rho> = 1), periodic on an N^3 grid (FFT-generated)."""
    try:
        import scipy.fft as sfft
        rfftn, irfftn = (lambda a: sfft.rfftn(a, workers=-1)), (lambda a, s: sfft.irfftn(a, s=s, workers=-1))
    except Exception:  # pragma: no cover
        rfftn, irfftn = np.fft.rfftn, (lambda a, s: np.fft.irfftn(a, s=s))
    white = g.standard_normal((N, N, N))
    wk = rfftn(white)
    kz = np.fft.fftfreq(N)[:, None, None]
    ky = np.fft.fftfreq(N)[None, :, None]
    kx = np.fft.rfftfreq(N)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kk[0, 0, 0] = 1.0
    amp = kk ** (slope / 2.0)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del kk, amp
    f = irfftn(wk, (N, N, N))
    del wk
    f -= f.mean()
    f *= sigma / f.std()
    f -= 0.5 * sigma * sigma
    return f


def config4(N=512, n_sub=100, precision="fp64", seed_offset=4):
    """3D throughput run: [0, 1)^3 periodic, N^3 cells; ln rho a k^{-11/3} Gaussian field with
    sigma_ln rho = 1 and <rho> = 1; T = exp(0.2 N(0,1)); v_i ~ N(0, (0.001 c)^2); absorption coefficients
    proportional to rho, kP = kF = 512 rho (k dx = rho at N = 512: optically thin to thick cells);
    E = a_R T^4 (1 + 0.1 U[-1,1]); F = c E f n with f ~ U[0, 0.5] and n isotropic; c = 10, chat = 1;
    FULL exchange, O(beta tau) on, theta = 1.  The gas speed keeps beta tau small in every cell, the
    regime in which the paper treats the O(beta tau) terms explicitly (Section 3.4)."""
    g = rng(seed_offset)
    dx = 1.0 / N
    desc = base_desc((N, N, N), (dx, dx, dx), bc="periodic", c=10.0, exchange="full", beta_tau=True,
                     kappa_P=512.0, kappa_F=512.0, kappa_rho_pow=1, theta_F=1.0, theta_E=1.0,
                     E_floor=1e-30, precision=precision)
    shp = (N, N, N)
    rho = np.exp(lognormal_field(N, g))
    T = np.exp(0.2 * g.standard_normal(shp))
    c = desc["c"]
    vx = (0.001 * c) * g.standard_normal(shp)
    vy = (0.001 * c) * g.standard_normal(shp)
    vz = (0.001 * c) * g.standard_normal(shp)
    E = desc["a_rad"] * T ** 4 * (1.0 + 0.1 * g.uniform(-1.0, 1.0, size=shp))
    f = g.uniform(0.0, 0.5, size=shp)
    nx_, ny_, nz_ = random_directions(g, shp)
    fields = {
        "E": E, "Fx": c * E * f * nx_, "Fy": c * E * f * ny_, "Fz": c * E * f * nz_,
        "T": T, "rho": rho, "vx": vx, "vy": vy, "vz": vz, "kP": None, "kF": None, "j": None,
    }
    return {"name": f"config4_throughput{N}", "desc": desc, "fields": fields, "chat": 1.0,
            "dt": cfl_dt(desc, 1.0), "n_sub": n_sub}


def config5(n_grids=64, sizes=(32, 48, 64, 96, 128), n_sub=50, precision="split", seed_offset=5):
    """Batched ensemble: n_grids independent grids on [-0.5, 0.5]^3 with N drawn from `sizes`, outflow,
    each with its own Gaussian source luminosity L ~ logU(1e-2, 1e2) (width 0.05) and uniform opacity
    tau ~ logU(0.1, 1000) per box length; FULL exchange, theta = 1, c = 10 chat, chat = 1,
    dt = 0.4 dx / chat per grid.  Gas at rest, rho = 1, T = 1, E = a_R T^4, F = 0."""
    g = rng(seed_offset)
    cases = []
    Ns = g.choice(np.array(sizes), size=n_grids)
    Ls = np.exp(g.uniform(math.log(1e-2), math.log(1e2), size=n_grids))
    taus = np.exp(g.uniform(math.log(0.1), math.log(1000.0), size=n_grids))
    for i in range(n_grids):
        N = int(Ns[i])
        dx = 1.0 / N
        desc = base_desc((N, N, N), (dx, dx, dx), bc="outflow", c=10.0, exchange="full", beta_tau=False,
                         kappa_P=float(taus[i]), kappa_F=float(taus[i]), kappa_rho_pow=0, theta_F=1.0,
                         theta_E=1.0, E_floor=1e-30, precision=precision)
        X, Y, Z = cell_centres(desc, x0=(-0.5, -0.5, -0.5))
        r2 = X ** 2 + Y ** 2 + Z ** 2
        sig = 0.05
        j = float(Ls[i]) * np.exp(-r2 / (2 * sig ** 2)) / (2 * math.pi * sig ** 2) ** 1.5
        shp = X.shape
        fields = {
            "E": np.ones(shp), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
            "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None,
            "kP": None, "kF": None, "j": j,
        }
        cases.append({"name": f"config5_grid{i}_N{N}", "desc": desc, "fields": fields, "chat": 1.0,
                      "dt": cfl_dt(desc, 1.0), "n_sub": n_sub})
    return cases


# ----------------------------------------------------------------------------- non-equilibrium Marshak wave

def marshak_case(N, eps=1.0, precision="fp64", chi_max=100.0, F_inc=0.25, E_floor=1e-10):
    """Section 4.1.4: a cold, static, absorbing slab chi = sqrt(3) rho kappa_0 x in [0, chi_max] with
    rho = kappa_0 = 1, a_R = c = chat = 1, F_inc = 1/4 (so u = E and v = T^4), the linear exchange
    of the Pomraning material with retardation eps, theta = 1.  E = E_floor and T = 0 initially (the
    cold medium; E > 0 keeps the closure defined), F = 0.  The low x face is the Marshak boundary
    (set before every subcycle from the Su & Olson surface value), the high face the Dirichlet state
    (E_floor, 0).  tau = eps c rho kappa_0 t = eps t."""
    L = chi_max / math.sqrt(3.0)
    desc = base_desc((N, 1, 1), (L / N, 1.0, 1.0), bc="dirichlet", c=1.0, exchange="linear", kappa_P=1.0,
                     kappa_F=1.0, kappa_rho_pow=1, theta_F=1.0, theta_E=1.0, E_floor=E_floor, precision=precision)
    desc["linear_eps"] = float(eps)
    desc["dirichlet_hi"] = [[E_floor, 0.0, 0.0, 0.0] for _ in range(3)]
    desc["dirichlet_lo"] = [[E_floor, 0.0, 0.0, 0.0] for _ in range(3)]
    shp = (1, 1, N)
    fields = {"E": np.full(shp, E_floor), "Fx": np.zeros(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
              "T": np.zeros(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None, "kP": None, "kF": None,
              "j": None}
    dt = desc["cfl"] * (L / N) / 1.0
    return {"name": f"marshak_{N}", "desc": desc, "fields": fields, "chat": 1.0, "dt": dt, "n_sub": 1,
            "marshak": {"eps": float(eps), "F_inc": F_inc, "tau_rate": float(eps) * 1.0 * 1.0 * 1.0}}


def marshak_subcycles(tau_end, case):
    """Subcycles of length case['dt'] that reach tau_end (the last one may end past it)."""
    return int(math.ceil(tau_end / (case["marshak"]["tau_rate"] * case["dt"]) - 1e-12))
