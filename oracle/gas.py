"""Plain FP64 NumPy oracle of the gas step around the radiation subcycles (Section 3.1 steps 3 and 6,
Section 3.4's closing paragraphs).  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
benchmark's CPU-baseline leg use it; the product library never does, and it shares no code with the
CUDA path.

What it computes, in the paper's order:

  * the gas subsystem of Eq. (algorithm:gastransport): the Euler equations for (rho, rho v, E_gas)
    with the explicit gas sources S_e,gas of Eq. (algorithm:source:explicit:gas) and no gravity
    (Phi = 0).  With k_F = rho kappa_0 and G = F/c those sources are
        rho v row:  k_F (G - (4/3) (v/c) E)
        E_gas row:  -k_F v . G
    (the terms with v are the O(beta tau) terms and are dropped when beta_tau is off);
  * one gas step of the van Leer predictor / corrector integrator (Section 3.4): a first-order
    predictor over dt/2 whose sources use the gas and the radiation at t^n, then a second-order
    corrector over dt with piecewise-linear reconstruction whose sources use the gas at t^{n+1/2}
    and the radiation still at t^n;
  * after the radiation subcycles, the correction of the sources to second order,
        dt/2 [S_e,gas(U_gas^{n+1/2}, U_rad^{n+1}) - S_e,gas(U_gas^{n+1/2}, U_rad^n)].

Readings where the paper leaves the hydrodynamics to its host code:
  * Riemann solver: HLLC (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Sec. 10.4)
    with the Davis wave-speed estimates S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R);
    the left star state is used when S* = 0; where the contact-speed denominator is not negative
    (zero pressure on both sides of a diverging face) the HLL flux is used instead;
  * reconstruction: primitive variables (rho, v, P), limited slopes componentwise with the grid's
    limiter (minmod, MC or none, as for the radiation); if either face value of a cell has rho <= 0 or
    P <= 0, that cell's slope in that direction is zeroed;
  * ghost cells: the ghost rule of the radiation path, applied per direction x, y, z (periodic wraps,
    outflow and Dirichlet faces take the nearest cell, reflect mirrors and negates the normal velocity
    and the normal G); the predictor is applied on two ghost layers of the ghost-filled state, and the
    gas sources there see the radiation through the same rule;
  * internal energy floor: a negative internal energy after a stage is set to zero (counted);
  * P = rho T / (mu/k_B), e = P / (gamma - 1), E_gas = e + rho |v|^2 / 2.

Arrays are float64 with shape (nz, ny, nx); the grid description is the dict of the seeded input
generators (n, dx, bc_lo, bc_hi, gamma, mu_over_kB, c, kappa_F, kappa_rho_pow, limiter, beta_tau).
"""
from __future__ import annotations

import numpy as np

GHOST = 2  # ghost layers of the predictor's half-step state (the corrector's stencil is i-2 .. i+1)


# ----------------------------------------------------------------------------- ghost cells

def axis_map(n, g, lo, hi, c0=None, c1=None):
    """Interior index and sign of the normal component for the coordinates -g .. n+g-1 of one axis
    (or c0 .. c1-1 when given)."""
    idx, sgn = [], []
    for c in range(-g if c0 is None else c0, n + g if c1 is None else c1):
        s = 1.0
        while c < 0 or c >= n:
            low = c < 0
            bc = lo if low else hi
            if bc == "periodic":
                c %= n
            elif bc in ("outflow", "dirichlet"):
                c = 0 if low else n - 1
            elif bc == "reflect":
                c = -c - 1 if low else 2 * n - 1 - c
                s = -s
            else:
                raise ValueError(bc)
        idx.append(c)
        sgn.append(s)
    return np.array(idx), np.array(sgn)


def with_ghosts(desc, a, g, normal=None, box=None):
    """The array a extended by g ghost layers in every active direction (or, with box = (lo, hi), the
    cells lo - g .. hi + g - 1 of the grid extended so).  normal = d marks a vector component along d,
    whose sign flips where the direction d is mirrored."""
    out = a
    for d in range(3):
        n = desc["n"][d]
        if n <= 1:
            continue
        lo, hi = (0, n) if box is None else (box[0][d], box[1][d])
        idx, sgn = axis_map(n, g, desc["bc_lo"][d], desc["bc_hi"][d], lo - g, hi + g)
        out = np.take(out, idx, axis=2 - d)
        if normal == d:
            shape = [1, 1, 1]
            shape[2 - d] = len(sgn)
            out = out * sgn.reshape(shape)
    return out


# ----------------------------------------------------------------------------- state conversions

def pressure(desc, rho, T):
    return rho * T / desc["mu_over_kB"]


def conserved(desc, W):
    """(rho, vx, vy, vz, P) -> (rho, Mx, My, Mz, E_gas)."""
    rho, vx, vy, vz, P = W
    e = P / (desc["gamma"] - 1.0)
    return [rho, rho * vx, rho * vy, rho * vz, e + 0.5 * rho * (vx * vx + vy * vy + vz * vz)]


def primitive(desc, U):
    """(rho, Mx, My, Mz, E_gas) -> (rho, vx, vy, vz, P) and the mask of cells whose internal energy
    was negative (floored to zero)."""
    rho, Mx, My, Mz, Eg = U
    vx, vy, vz = Mx / rho, My / rho, Mz / rho
    e = Eg - 0.5 * (Mx * vx + My * vy + Mz * vz)
    neg = e < 0.0
    e = np.where(neg, 0.0, e)
    return [rho, vx, vy, vz, (desc["gamma"] - 1.0) * e], neg


def temperature(desc, rho, P):
    return P * desc["mu_over_kB"] / rho


# ----------------------------------------------------------------------------- fluxes

def euler_flux(W, d, gamma):
    """Flux of (rho, Mx, My, Mz, E_gas) in direction d of the primitive state W."""
    rho, P = W[0], W[4]
    v = W[1:4]
    u = v[d]
    Eg = P / (gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    F = [rho * u, rho * v[0] * u, rho * v[1] * u, rho * v[2] * u, (Eg + P) * u]
    F[1 + d] = F[1 + d] + P
    return F, Eg


def hllc(WL, WR, d, gamma):
    """HLLC flux (Toro Sec. 10.4) between the primitive states WL, WR across a face normal to d."""
    FL, EL = euler_flux(WL, d, gamma)
    FR, ER = euler_flux(WR, d, gamma)
    rL, uL, PL = WL[0], WL[1 + d], WL[4]
    rR, uR, PR = WR[0], WR[1 + d], WR[4]
    aL = np.sqrt(gamma * PL / rL)
    aR = np.sqrt(gamma * PR / rR)
    SL = np.minimum(uL - aL, uR - aR)
    SR = np.maximum(uL + aL, uR + aR)
    den = rL * (SL - uL) - rR * (SR - uR)
    with np.errstate(divide="ignore", invalid="ignore"):
        Ss = (PR - PL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / den

        def star(W, E, S, F):
            r, u, P = W[0], W[1 + d], W[4]
            chi = r * (S - u) / (S - Ss)
            Us = [chi, chi * W[1], chi * W[2], chi * W[3], chi * (E / r + (Ss - u) * (Ss + P / (r * (S - u))))]
            Us[1 + d] = chi * Ss
            U = conserved_from(W, E)
            return [F[q] + S * (Us[q] - U[q]) for q in range(5)]

        FsL = star(WL, EL, SL, FL)
        FsR = star(WR, ER, SR, FR)
        UL = conserved_from(WL, EL)
        UR = conserved_from(WR, ER)
        Fhll = [(SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) / (SR - SL) for q in range(5)]
    out = []
    for q in range(5):
        mid = np.where(Ss >= 0.0, FsL[q], FsR[q])
        mid = np.where(den < 0.0, mid, Fhll[q])
        out.append(np.where(SL >= 0.0, FL[q], np.where(SR <= 0.0, FR[q], mid)))
    return out


def conserved_from(W, E):
    rho = W[0]
    return [rho, rho * W[1], rho * W[2], rho * W[3], E]


# ----------------------------------------------------------------------------- reconstruction

def limited_slope(dl, dr, limiter):
    if limiter == "none":
        return 0.5 * (dl + dr)
    s = np.where(dl > 0.0, 1.0, -1.0)
    a, b = np.abs(dl), np.abs(dr)
    if limiter == "minmod":
        m = np.minimum(a, b)
    elif limiter == "mc":
        m = np.minimum(2.0 * np.minimum(a, b), 0.5 * np.abs(dl + dr))
    else:
        raise ValueError(limiter)
    return np.where(dl * dr <= 0.0, 0.0, s * m)


def shift(a, d, k):
    """a[i + k e_d] for the array a (numpy axis 2 - d), cropped later by the caller."""
    return np.roll(a, -k, axis=2 - d)


# ----------------------------------------------------------------------------- sources

def absorption_F(desc, rho, kF):
    if kF is not None:
        return kF
    p = int(desc["kappa_rho_pow"])
    kap = desc["kappa_F"]
    return kap if p == 0 else (kap * rho if p == 1 else (kap * rho) * rho)


def gas_source(desc, k, v, E, G):
    """S_e,gas of Eq. (algorithm:source:explicit:gas) with Phi = 0: the rho v and E_gas rows."""
    c = desc["c"]
    bt = bool(desc["beta_tau"])
    SM = [k * (G[a] - (4.0 / 3.0) * v[a] * E / c) if bt else k * G[a] for a in range(3)]
    SE = -k * (v[0] * G[0] + v[1] * G[1] + v[2] * G[2]) if bt else 0.0 * k
    return SM, SE


# ----------------------------------------------------------------------------- the step

def active(desc):
    return [desc["n"][d] > 1 for d in range(3)]


def crop(desc, a, g):
    """The interior of an array that carries g ghost layers in each active direction."""
    sl = []
    for d in (2, 1, 0):
        sl.append(slice(g, g + desc["n"][d]) if desc["n"][d] > 1 else slice(None))
    return a[tuple(sl)]


def gas_step(desc, gas, rad, dt, box=None):
    """One gas step over dt.  gas: dict rho, vx, vy, vz, T (vx.. may be None: zero), optional kF;
    rad: dict E, Fx, Fy, Fz (F in flux units).  Returns (gas at t^{n+1} before the source
    correction, pending data for gas_correct, number of floored cells).  With box = (lo, hi) only the
    cells lo <= (x, y, z) < hi are computed and returned (the same arithmetic on the cells they
    depend on)."""
    c = desc["c"]
    shp = gas["rho"].shape
    v = [gas.get(k) if gas.get(k) is not None else np.zeros(shp) for k in ("vx", "vy", "vz")]
    kF = gas.get("kF")
    W = [gas["rho"], v[0], v[1], v[2], pressure(desc, gas["rho"], gas["T"])]
    E = rad["E"]
    G = [rad["Fx"] / c, rad["Fy"] / c, rad["Fz"] / c]

    # (1) ghost-filled state at t^n: three layers, so that the predictor can be applied on two
    g3 = GHOST + 1
    Wg = [with_ghosts(desc, W[0], g3, box=box), with_ghosts(desc, W[1], g3, 0, box),
          with_ghosts(desc, W[2], g3, 1, box), with_ghosts(desc, W[3], g3, 2, box), with_ghosts(desc, W[4], g3, box=box)]
    Eg3 = with_ghosts(desc, E, g3, box=box)
    Gg3 = [with_ghosts(desc, G[a], g3, a, box) for a in range(3)]
    kFg3 = None if kF is None else with_ghosts(desc, kF, g3, box=box)
    if box is not None:
        # the box is the grid of the steps below; its ghost layers are the neighbouring cells
        desc = dict(desc, n=tuple(box[1][d] - box[0][d] if desc["n"][d] > 1 else 1 for d in range(3)))
        sl = tuple(slice(box[0][d], box[1][d]) for d in (2, 1, 0))
        W = [w[sl] for w in W]
        E = E[sl]
        G = [g[sl] for g in G]
        kF = None if kF is None else kF[sl]
        shp = W[0].shape
    return _step(desc, dt, W, E, G, kF, Wg, Eg3, Gg3, kFg3, shp)


def _step(desc, dt, W, E, G, kF, Wg, Eg3, Gg3, kFg3, shp):
    gam = desc["gamma"]
    act = active(desc)
    g3 = GHOST + 1
    floors = 0

    # (2) predictor: first-order HLLC fluxes and the half step (sources from U_gas^n, U_rad^n)
    Ug = conserved(desc, Wg)
    dU = [np.zeros_like(Wg[0]) for _ in range(5)]
    for d in range(3):
        if not act[d]:
            continue
        WL = [shift(w, d, -1) for w in Wg]  # the cell on the low side of face i - 1/2
        F = hllc(WL, Wg, d, gam)            # F[i] = flux through face i - 1/2
        for q in range(5):
            dU[q] -= (shift(F[q], d, 1) - F[q]) / desc["dx"][d]
    SM, SE = gas_source(desc, absorption_F(desc, Wg[0], kFg3), Wg[1:4], Eg3, Gg3)
    S = [0.0 * SE, SM[0], SM[1], SM[2], SE]
    Uh = [Ug[q] + 0.5 * dt * dU[q] + 0.5 * dt * S[q] for q in range(5)]
    # keep two ghost layers (the outermost layer's fluxes used wrapped neighbours: discarded)
    Uh = [crop_to(desc, u, g3, GHOST) for u in Uh]
    Wh, neg = primitive(desc, Uh)
    floors += int(np.count_nonzero(neg[interior_mask(desc, GHOST)]))

    # (3) corrector: limited piecewise-linear primitives of the half-step state, HLLC, full step
    lim = desc["limiter"]
    dU = [np.zeros_like(Wh[0]) for _ in range(5)]
    for d in range(3):
        if not act[d]:
            continue
        slope = [limited_slope(w - shift(w, d, -1), shift(w, d, 1) - w, lim) for w in Wh]
        bad = np.zeros(Wh[0].shape, dtype=bool)
        for sgn in (-0.5, 0.5):
            bad |= ~(Wh[0] + sgn * slope[0] > 0.0) | ~(Wh[4] + sgn * slope[4] > 0.0)
        slope = [np.where(bad, 0.0, s) for s in slope]
        WR = [Wh[q] - 0.5 * slope[q] for q in range(5)]                                  # cell i, low face
        WL = [shift(Wh[q], d, -1) + 0.5 * shift(slope[q], d, -1) for q in range(5)]    # cell i-1, high face
        F = hllc(WL, WR, d, gam)
        for q in range(5):
            dU[q] -= (shift(F[q], d, 1) - F[q]) / desc["dx"][d]
    dU = [crop(desc, u, GHOST) for u in dU]
    Whi = [crop(desc, w, GHOST) for w in Wh]
    kh = absorption_F(desc, Whi[0], kF)
    SM, SE = gas_source(desc, kh, Whi[1:4], E, G)
    S = [0.0 * SE, SM[0], SM[1], SM[2], SE]
    U0 = conserved(desc, W)
    U1 = [U0[q] + dt * dU[q] + dt * S[q] for q in range(5)]
    W1, neg = primitive(desc, U1)
    floors += int(np.count_nonzero(neg))
    out = {"rho": W1[0], "vx": W1[1], "vy": W1[2], "vz": W1[3], "T": temperature(desc, W1[0], W1[4])}
    pending = {"dt": dt, "kF": kh * np.ones(shp), "v": [Whi[1], Whi[2], Whi[3]], "E": E, "G": G}
    return out, pending, floors


def crop_to(desc, a, g_have, g_keep):
    sl = []
    for d in (2, 1, 0):
        if desc["n"][d] > 1:
            o = g_have - g_keep
            sl.append(slice(o, o + desc["n"][d] + 2 * g_keep))
        else:
            sl.append(slice(None))
    return a[tuple(sl)]


def interior_mask(desc, g):
    shape = [desc["n"][d] + 2 * g if desc["n"][d] > 1 else 1 for d in (2, 1, 0)]
    m = np.zeros(shape, dtype=bool)
    m[tuple(slice(g, g + desc["n"][d]) if desc["n"][d] > 1 else slice(None) for d in (2, 1, 0))] = True
    return m


def gas_correct(desc, gas, pending, rad):
    """The second-order correction of the gas sources with the radiation at t^{n+1} (rad), applied to
    the gas returned by gas_step.  Returns (gas, number of floored cells)."""
    c = desc["c"]
    dt = pending["dt"]
    W = [gas["rho"], gas["vx"], gas["vy"], gas["vz"], pressure(desc, gas["rho"], gas["T"])]
    U = conserved(desc, W)
    G1 = [rad["Fx"] / c, rad["Fy"] / c, rad["Fz"] / c]
    SM1, SE1 = gas_source(desc, pending["kF"], pending["v"], rad["E"], G1)
    SM0, SE0 = gas_source(desc, pending["kF"], pending["v"], pending["E"], pending["G"])
    for a in range(3):
        U[1 + a] = U[1 + a] + 0.5 * dt * (SM1[a] - SM0[a])
    U[4] = U[4] + 0.5 * dt * (SE1 - SE0)
    W1, neg = primitive(desc, U)
    out = {"rho": W1[0], "vx": W1[1], "vy": W1[2], "vz": W1[3], "T": temperature(desc, W1[0], W1[4])}
    return out, int(np.count_nonzero(neg))


# ----------------------------------------------------------------------------- step 2 (option)

def gas_exchange(desc, gas, rad, dt, chat):
    """Section 3.1 step 2 for the option that integrates the stiff exchange S_i (Eq.
    algorithm:source:implicit) once per gas step: the implicit gas-radiation energy exchange over dt =
    Delta t_gas in every cell (the quartic theta scheme of Eqs. source:energyupdate - source:polynomial,
    the radiation oracle's cell routine), on E floored at E_floor, followed by |F| <= cE (the order of
    the per-subcycle exchange).  k_P is the kP array or kappa_P rho^p.  Returns (gas with the new T,
    radiation with the new E and F, number of theta = 1 fallbacks)."""
    from . import oracle as orc

    c = desc["c"]
    E = np.array(rad["E"], dtype=np.float64, copy=True)
    F = [np.array(rad[k], dtype=np.float64, copy=True) for k in ("Fx", "Fy", "Fz")]
    T = np.array(gas["T"], dtype=np.float64, copy=True)
    rho = gas["rho"]
    kP = gas.get("kP")
    if kP is None:
        p = int(desc["kappa_rho_pow"])
        kap = desc["kappa_P"]
        kP = kap * np.ones_like(rho) if p == 0 else (kap * rho if p == 1 else (kap * rho) * rho)
    fallbacks = 0
    for i in np.ndindex(E.shape):
        Ei = max(float(E[i]), desc["E_floor"])
        Ei, Ti, fb = orc.exchange_full(desc, chat, dt, float(rho[i]), float(kP[i]), Ei, float(T[i]))
        E[i], T[i] = Ei, Ti
        fallbacks += fb
        g2 = (F[0][i] / c) ** 2 + (F[1][i] / c) ** 2 + (F[2][i] / c) ** 2
        if g2 > Ei * Ei:
            s = Ei / np.sqrt(g2)
            for a in range(3):
                F[a][i] *= s
    return dict(gas, T=T), {"E": E, "Fx": F[0], "Fy": F[1], "Fz": F[2]}, fallbacks
