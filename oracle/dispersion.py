"""Linear waves of the coupled radiation-hydrodynamics system under the reduced speed of light
approximation (Section 4.3.1, "RHD Linear Waves"): the temporal dispersion relation (the initial value
problem, Eq. radlinearwave:ivp:dispersion), its modes and their eigenvectors, and the initial state of a
single mode for a simulation.  TEST INFRASTRUCTURE: the checker of the linear-wave runs (the oracle's
and the library's); the product library never uses it.

Units are those of the paper's analysis: density rho_0 = 1, wavelength lambda = 1, adiabatic sound
speed a_0 = 1 (time unit lambda / a_0), background at rest in radiative equilibrium, T_0 = 1.  The
parameters are P_0 = a_R T_0^4 / (rho_0 a_0^2), C = c / a_0, Chat = chat / a_0 and the optical depth per
wavelength tau = rho_0 kappa_0 lambda; gamma is the adiabatic index.  A grid description with these units
has mu_over_kB = gamma (so that a_0^2 = gamma T_0 / (mu/k_B) = 1), a_R = P_0, c = C, kappa_P = kappa_F = tau
with absorption coefficients proportional to rho, and the Eddington closure (P1).

Modes.  The linearised equations (Eqs. mixedframe:graysystem with 1/chat in front of the radiation time
derivatives and the Eddington tensor I/3) for a perturbation exp(i (k x - omega t)) with k = 2 pi of
(delta rho, delta v, delta T, delta E, delta F / c) read

    -i w drho + i k dv                                                      = 0
    -i w dv + i k (drho + dT) / gamma                                       = tau df - (4/3) tau P_0 dv / C
    -i w (drho + dT) / (gamma (gamma - 1)) + i k dv / (gamma - 1)           = -C tau (4 P_0 dT - dE)
    -i w dE / Chat + i k df                                                 = tau (4 P_0 dT - dE)
    -i w df / Chat + i k dE / 3                                             = -tau df + (4/3) tau P_0 dv / C

(mass, gas momentum, gas energy with e = P / (gamma - 1), radiation energy, radiation flux; the terms in
v/c of the momentum equations are those of the paper's system).  With omega = 2 pi Z they form a
generalised eigenvalue problem A x = i omega B x whose five eigenvalues are the roots of the quintic
Eq. (radlinearwave:ivp:dispersion) up to terms of order P_0 tau / C that the quintic leaves out, with the
reading that its last bracket carries Chat (the printed text has C there; the equations above give
Chat, and only then is the radiation-modified acoustic mode affected by the RSLA, as the paper states).
"""
from __future__ import annotations

import math

import numpy as np


def _matrices(P0, C, Ch, tau, gamma):
    """A, B with the linear system M(omega) = A - i omega B (rows: the five equations above)."""
    k = 2.0 * math.pi
    g = gamma
    A = np.zeros((5, 5), dtype=complex)
    B = np.zeros((5, 5), dtype=complex)
    # unknowns: drho, dv, dT, dE, df
    A[0, 1] = 1j * k
    B[0, 0] = 1.0
    A[1, 0] = 1j * k / g
    A[1, 2] = 1j * k / g
    A[1, 1] = (4.0 / 3.0) * tau * P0 / C
    A[1, 4] = -tau
    B[1, 1] = 1.0
    A[2, 1] = 1j * k / (g - 1.0)
    A[2, 2] = C * tau * 4.0 * P0
    A[2, 3] = -C * tau
    B[2, 0] = 1.0 / (g * (g - 1.0))
    B[2, 2] = 1.0 / (g * (g - 1.0))
    A[3, 2] = -tau * 4.0 * P0
    A[3, 3] = tau
    A[3, 4] = 1j * k
    B[3, 3] = 1.0 / Ch
    A[4, 1] = -(4.0 / 3.0) * tau * P0 / C
    A[4, 3] = 1j * k / 3.0
    A[4, 4] = tau
    B[4, 4] = 1.0 / Ch
    return A, B


def linear_modes(P0, C, Ch, tau, gamma=5.0 / 3.0):
    """The five modes: (Z, X) with Z = omega / (a_0 k) (sorted by real part) and the columns of X the
    eigenvectors (delta rho, delta v, delta T, delta E, delta F / c)."""
    A, B = _matrices(P0, C, Ch, tau, gamma)
    lam, X = np.linalg.eig(np.linalg.solve(B, A))   # A x = lam B x, lam = i omega
    Z = -1j * lam / (2.0 * math.pi)
    order = np.argsort(Z.real)
    return Z[order], X[:, order]


def ivp_quintic(P0, C, Ch, tau, gamma=5.0 / 3.0, last_bracket=None):
    """Coefficients (highest degree first) of the quintic Eq. (radlinearwave:ivp:dispersion) in Z.
    last_bracket: the speed in the last bracket's two terms (default Chat, the reading above; pass C for
    the printed text)."""
    g = gamma
    cl = Ch if last_bracket is None else last_bracket
    P = np.polynomial.Polynomial
    Zp = P([0.0, 1.0])
    a = 1j * Ch * tau / (2.0 * math.pi)
    t1 = (Zp ** 2 - 1) * Zp * (1 - (3.0 / Ch ** 2) * (Zp + a) ** 2 - 1j * (2 * g * P0 * tau / (math.pi * Ch)) * (Zp + a))
    t2 = 1j * (2 * (g - 1) * P0 * C * tau / math.pi) * (g * Zp ** 2 - 1) * (
        1 - (3.0 / Ch ** 2) * (1 - Ch / (3 * (g - 1) * C)) * Zp * (Zp + a))
    t3 = 1j * (2 * (g - 1) * P0 * tau / (math.pi * Ch)) * Zp * (
        1j * 2 * g * P0 * cl * tau / (3 * math.pi) + Zp / (3 * (g - 1)) + 1j * cl * tau / (2 * math.pi))
    return (t1 + t2 + t3).coef[::-1]


def newton_root(coeffs, Z0, tol=1e-14, max_iter=100):
    """A root of the polynomial (coefficients highest degree first) by Newton-Raphson from Z0."""
    p = np.poly1d(coeffs)
    dp = p.deriv()
    Z = complex(Z0)
    for _ in range(max_iter):
        step = p(Z) / dp(Z)
        Z -= step
        if abs(step) <= tol * max(1.0, abs(Z)):
            break
    return Z


def acoustic_mode(P0, C, Ch, tau, gamma=5.0 / 3.0):
    """(Z, x) of the acoustic mode travelling in +x: of the modes with 0 < Re Z < max(1, a_0*) + 0.5 (the
    radiation modes travel near Chat / sqrt(3)), the least damped."""
    Z, X = linear_modes(P0, C, Ch, tau, gamma)
    a_star = radiation_acoustic_speed(P0, gamma)
    cand = [j for j in range(5) if 0.05 < Z[j].real < max(1.0, a_star) + 0.5]
    j = min(cand, key=lambda q: abs(Z[q].imag))
    return Z[j], X[:, j]


def radiation_acoustic_speed(P0, gamma=5.0 / 3.0):
    """a_0* / a_0, the radiation-modified acoustic speed (Eq. radlinearwave:radiationacousticspeed)."""
    g = gamma
    return math.sqrt((9 + 60 * P0 * (g - 1) + 16 * P0 ** 2 * g * (g - 1)) / (1 + 4 * P0 * g * (g - 1))) / 3.0


def mode_state(N, P0, C, Ch, tau, gamma=5.0 / 3.0, amplitude=1e-6, mode=None):
    """Fields (rho, T, vx, E, Fx as arrays of shape (1, 1, N)) of the periodic unit box holding one
    wavelength of a mode at point values of the cell centres, with max |delta rho| = amplitude; and the
    mode's Z.  mode = (Z, x) (default: the acoustic mode)."""
    Z, x = acoustic_mode(P0, C, Ch, tau, gamma) if mode is None else mode
    x = x / x[0] * amplitude
    X = (np.arange(N) + 0.5) / N
    ph = np.exp(2j * math.pi * X)
    f = lambda q: np.ascontiguousarray((x[q] * ph).real).reshape(1, 1, N)
    return {"rho": 1.0 + f(0), "vx": f(1), "T": 1.0 + f(2), "E": P0 + f(3), "Fx": C * f(4)}, Z


def measured_Z(times, drho):
    """Z of the k = 2 pi Fourier amplitude of delta rho(x, t) (rows: times), with the phase unwrapped in
    time: a least-squares fit of log A(t) = log A(0) - i 2 pi Z t."""
    t = np.asarray(times, dtype=float)
    N = drho.shape[1]
    X = (np.arange(N) + 0.5) / N
    A = (np.asarray(drho) * np.exp(-2j * math.pi * X)).sum(axis=1) * (2.0 / N)
    phase = np.unwrap(np.angle(A))
    logm = np.log(np.abs(A))
    sr = np.polyfit(t, phase, 1)[0]   # d phase / dt = -Re omega
    si = np.polyfit(t, logm, 1)[0]    # d log |A| / dt = Im omega
    return complex(-sr, si) / (2.0 * math.pi)
