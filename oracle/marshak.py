"""The non-equilibrium Marshak wave of Section 4.1.4 (test infrastructure only): the Su & Olson
surface value u(0, tau) that sets the left boundary, and the boundary state it gives.  Plain FP64
numpy, written from the paper's Eq. (marshak:suolson) at chi = 0 and Eq. (marshak:bc_ix1); shares no
code with the CUDA path.

At chi = 0 the sines reduce to sin(Theta_n) = 2 Gamma_n / sqrt(3 + 4 Gamma_n^2), since
cos(Theta_n) = sqrt(3 / (3 + 4 Gamma_n^2)).  The two integrals over eta in (0, 1) are taken by the
midpoint rule, as the paper does (n points).
"""
import math

import numpy as np


def gamma1(eta, eps):
    return eta * np.sqrt(eps + 1.0 / (1.0 - eta * eta))


def gamma2(eta, eps):
    return np.sqrt((1.0 - eta) * (eps + 1.0 / eta))


def surface_u(tau, eps, n=4096):
    """u(0, tau) = c E(0, t) / (4 F_inc) of Eq. (marshak:suolson), midpoint rule with n points."""
    eta = (np.arange(n, dtype=np.float64) + 0.5) / n
    g1 = gamma1(eta, eps)
    th1 = np.arccos(np.sqrt(3.0 / (3.0 + 4.0 * g1 * g1)))
    i1 = np.exp(-tau * eta * eta) * np.sin(th1) / (eta * np.sqrt(3.0 + 4.0 * g1 * g1))
    g2 = gamma2(eta, eps)
    th2 = np.arccos(np.sqrt(3.0 / (3.0 + 4.0 * g2 * g2)))
    i2 = np.exp(-tau / (eps * eta)) * np.sin(th2) / (eta * (1.0 + eps * eta) * np.sqrt(3.0 + 4.0 * g2 * g2))
    s3 = math.sqrt(3.0)
    return 1.0 - (2.0 * s3 / math.pi) * np.sum(i1) / n - (s3 / math.pi) * math.exp(-tau) * np.sum(i2) / n


def boundary_state(tau, eps, F_inc, c, n=4096):
    """(E, F) at x = 0: E from u(0, tau), F from c E + 2 F = 4 F_inc (Eq. marshak:bc_ix1)."""
    E = 4.0 * F_inc * surface_u(tau, eps, n) / c
    return E, (4.0 * F_inc - c * E) / 2.0
