"""Reduced-speed-of-light time-step helpers, plain FP64 numpy (test infrastructure only).

Only the test-suite imports this module.  It states, as directly as the paper does, how the gas
signal speed, the radiation time step and the reduced speed of light are chosen (Section 3.1 and
Section 3.2 of Skinner & Ostriker 2013).  It shares no code with the CUDA path.

Readings (the paper leaves them open):
- kappa_0 of Eq. algorithm:ceff is taken as the flux-mean absorption coefficient k_F = rho kappa_F
  (the paper sets kappa_P = kappa_F = kappa_0), per cell from the kF array if given, else from the
  opacity law kappa_F rho^p.
- Delta x of Eqs. algorithm:ceff, algorithm:gastimestep and algorithm:radtimestep is the smallest
  spacing over the active directions.
- P = rho T / (mu / k_B) (the ideal gas of Eq. mixedframe:fullsystem with the descriptor's units).
- The maximum optical depth of Eq. rsla:diffcrit, when measured on a grid, is the largest sum of
  k_F Delta x_d along any grid line parallel to an active axis (the domain's optical depth along
  the axes).
- The number of subcycles per gas step ("about R", Section 3.1 step 5) is the smallest n with
  Delta t_gas / n <= K_0 Delta x / chat, and the subcycle length is Delta t_gas / n, so that n
  subcycles end exactly at t + Delta t_gas.
"""
import math

import numpy as np


def kappa_law(kappa, p, rho):
    """Absorption coefficient from the descriptor's opacity law: kappa rho^p, p in {0, 1, 2}."""
    if p == 0:
        return np.full_like(rho, kappa)
    if p == 1:
        return kappa * rho
    return (kappa * rho) * rho


def active_dx_min(desc):
    """Smallest cell spacing over the active directions (n > 1)."""
    return min(float(desc["dx"][d]) for d in range(3) if int(desc["n"][d]) > 1)


def flux_absorption(desc, fields):
    """k_F per cell (array of the fields' shape)."""
    kF = fields.get("kF")
    if kF is not None:
        return np.asarray(kF, dtype=np.float64)
    rho = np.asarray(fields["rho"], dtype=np.float64)
    return kappa_law(float(desc["kappa_F"]), int(desc["kappa_rho_pow"]), rho)


def effective_sound_speed(desc, fields, E):
    """Eq. algorithm:ceff: c_eff = sqrt((gamma P + (4/9) E (1 - exp(-k_F dx))) / rho) per cell."""
    rho = np.asarray(fields["rho"], dtype=np.float64)
    T = np.asarray(fields["T"], dtype=np.float64)
    P = rho * T / float(desc["mu_over_kB"])
    tau_cell = flux_absorption(desc, fields) * active_dx_min(desc)
    rad = (4.0 / 9.0) * np.asarray(E, dtype=np.float64) * (-np.expm1(-tau_cell))
    return np.sqrt((float(desc["gamma"]) * P + rad) / rho)


def max_signal_speed(desc, fields, E):
    """v_max = max over cells of |v| + c_eff (the definition under Eq. algorithm:gastimestep)."""
    speed = np.zeros_like(np.asarray(fields["rho"], dtype=np.float64))
    for k in ("vx", "vy", "vz"):
        v = fields.get(k)
        if v is not None:
            speed = speed + np.asarray(v, dtype=np.float64) ** 2
    return float(np.max(np.sqrt(speed) + effective_sound_speed(desc, fields, E)))


def max_optical_depth(desc, fields):
    """Largest line-integrated optical depth sum(k_F dx_d) over the grid lines along each active
    axis (arrays are indexed [z, y, x])."""
    kF = flux_absorption(desc, fields)
    best = 0.0
    for d in range(3):
        if int(desc["n"][d]) <= 1:
            continue
        axis = 2 - d
        line = np.sum(kF, axis=axis) * float(desc["dx"][d])
        best = max(best, float(np.max(line)))
    return best


def suggest_chat(c, v_max, tau_max, ratio):
    """Eq. rsla:staticdiffreq with 'much greater' read as the factor `ratio`:
    chat = ratio v_max max(1, tau_max), and chat = c where that is not below c (Section 3.1)."""
    return min(float(c), float(ratio) * float(v_max) * max(1.0, float(tau_max)))


def time_steps(cfl, dx_min, v_max, chat):
    """Eqs. algorithm:gastimestep and algorithm:radtimestep: dt_gas = K_0 dx / v_max, and the subcycle
    count n and length dt_gas / n (see the reading in the module header)."""
    dt_gas = float(cfl) * float(dx_min) / float(v_max)
    dt_max = float(cfl) * float(dx_min) / float(chat)
    n = max(1, int(math.ceil(dt_gas / dt_max)))
    while dt_gas / n > dt_max:
        n += 1
    return dt_gas, dt_gas / n, n
