"""Pins of the oracle's closure, wave speeds and HLL flux against what the paper and the
mathematics fix (Sections 2.3 and 3.3).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand_states(n, seed, fmin=0.0, fmax=1.0):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        E = float(np.exp(g.normal()))
        f = float(g.uniform(fmin, fmax))
        v = g.normal(size=3)
        v /= np.linalg.norm(v)
        out.append(np.array([E, *(E * f * v)]))
    return out


def test_chi_limits_and_range():
    # chi_at_f0, chi_at_f1, chi_range
    assert orc.chi(0.0) == pytest.approx(GOLD["chi_at_f0"]["value"], rel=1e-15)
    assert orc.chi(1.0) == pytest.approx(GOLD["chi_at_f1"]["value"], rel=1e-15)
    fs = np.linspace(0.0, 1.0, 2001)
    ch = np.array([orc.chi(f) for f in fs])
    assert np.all(np.diff(ch) > 0)
    lo, hi = GOLD["chi_range"]["value"]
    assert ch.min() >= lo - 1e-16 and ch.max() <= hi + 1e-16


def test_chi_equals_alternative_form():
    # chi_alt_form: the paper writes the same Eddington factor as (5 - 2 sqrt(4 - 3 f^2))/3
    for f in np.linspace(0.0, 1.0, 1001):
        alt = (5.0 - 2.0 * math.sqrt(4.0 - 3.0 * f * f)) / 3.0
        assert orc.chi(f) == pytest.approx(alt, rel=4e-16, abs=4e-16)


def test_eddington_tensor_conditions():
    # trace_T (Eq. m1:cond1) and the second sufficient condition (Eq. m1:cond2): T - f f >= 0
    for U in _rand_states(3000, 1):
        E, G = U[0], U[1:]
        T = orc.eddington_tensor(E, G)
        f = G / E
        assert np.trace(T) == pytest.approx(GOLD["trace_T"]["value"], abs=2e-15)
        assert np.allclose(T, T.T, atol=0)
        w = np.linalg.eigvalsh(T - np.outer(f, f))
        assert w.min() >= -1e-13
        # n is an eigenvector with eigenvalue chi(f)
        g = np.linalg.norm(G)
        if g > 0:
            n = G / g
            assert np.allclose(T @ n, orc.chi(min(g / E, 1.0)) * n, atol=1e-14)


def test_eddington_tensor_limits():
    # T_diffusion_limit, T_streaming_limit
    T0 = orc.eddington_tensor(2.0, [0.0, 0.0, 0.0])
    assert np.allclose(T0, np.eye(3) / 3.0, atol=1e-16)
    for U in _rand_states(50, 2):
        E = U[0]
        n = U[1:] / np.linalg.norm(U[1:])
        T1 = orc.eddington_tensor(E, E * n)
        assert np.allclose(T1, np.outer(n, n), atol=2e-15)
    assert np.allclose(orc.eddington_tensor(1.0, [0, 0, 0], closure="p1"), np.eye(3) / 3.0)


def test_division_free_pressure_form():
    """The CUDA path evaluates E T = (s-1)E/3 I + 3/(2+s) G G^T / E with s = sqrt(4 - 3 f^2), which
    is the paper's Eq. (m1:m1tns) rewritten with chi = (5 - 2 s)/3; both forms must agree."""
    for U in _rand_states(3000, 3):
        E, G = U[0], U[1:]
        f2 = float(G @ G) / (E * E)
        s = math.sqrt(4.0 - 3.0 * min(f2, 1.0))
        P_alt = (s - 1.0) * E / 3.0 * np.eye(3) + 3.0 / (2.0 + s) * np.outer(G, G) / E
        P_lit = E * orc.eddington_tensor(E, G)
        assert np.allclose(P_lit, P_alt, rtol=0, atol=8e-16 * E)


def test_wave_speed_limits():
    # evals_streaming_limit, evals_diffusion_limit
    chat = 3.7
    l1, l3 = orc.wave_speeds([1.5, 0, 0, 0], 0, chat)
    lo, _, hi = GOLD["evals_diffusion_limit"]["value"]
    assert l1 == pytest.approx(lo * chat, rel=1e-15)
    assert l3 == pytest.approx(hi * chat, rel=1e-15)
    for U in _rand_states(200, 4, fmin=1.0, fmax=1.0):
        E = U[0]
        n = U[1:] / np.linalg.norm(U[1:])
        for d in range(3):
            l1, l3 = orc.wave_speeds(U, d, chat)
            # the radicand is O(eps) at f = 1 up to rounding, so its root is O(sqrt(eps))
            assert l1 == pytest.approx(chat * n[d], abs=3e-8 * chat)
            assert l3 == pytest.approx(chat * n[d], abs=3e-8 * chat)
    l1, l3 = orc.wave_speeds([1.0, 0.3, 0.2, 0.1], 1, chat, speeds="fixed")
    assert (l1, l3) == (pytest.approx(-chat / math.sqrt(3)), pytest.approx(chat / math.sqrt(3)))


def test_wave_speed_ordering_with_lambda2():
    # evals_ordering with lambda_2 of Eq. (hyperbolic:evals2)
    chat = 1.0
    for U in _rand_states(4000, 5, fmin=1e-6, fmax=1.0):
        E, G = U[0], U[1:]
        f = np.linalg.norm(G) / E
        for d in range(3):
            mu = G[d] / np.linalg.norm(G)
            l2 = chat * (mu / f) * (2.0 - math.sqrt(4.0 - 3.0 * f * f))
            l1, l3 = orc.wave_speeds(U, d, chat)
            assert l1 <= l2 + 1e-12 and l2 <= l3 + 1e-12


def _jacobian(U, d, chat, h=1e-6):
    J = np.zeros((4, 4))
    for q in range(4):
        dU = np.zeros(4)
        dU[q] = h * max(abs(U[0]), 1.0)
        J[:, q] = (orc.flux(U + dU, d, chat) - orc.flux(U - dU, d, chat)) / (2 * dU[q])
    return J


def test_wave_speeds_are_jacobian_extremes():
    """lambda_1, lambda_3 (Eq. hyperbolic:evals13) must be the smallest and largest eigenvalue of
    the 4x4 flux Jacobian A = dF/dU (Eq. hyperbolic:linear), here by central differences."""
    chat = 2.0
    for U in _rand_states(300, 6, fmin=0.02, fmax=0.97):
        for d in range(3):
            w = np.linalg.eigvals(_jacobian(U, d, chat))
            assert np.max(np.abs(w.imag)) < 1e-5
            l1, l3 = orc.wave_speeds(U, d, chat)
            assert w.real.min() == pytest.approx(l1, abs=2e-6)
            assert w.real.max() == pytest.approx(l3, abs=2e-6)


def test_hll_consistency_and_upwinding():
    chat = 1.3
    for U in _rand_states(300, 7):
        for d in range(3):
            F = orc.flux(U, d, chat)
            assert np.allclose(orc.hll(U, U, d, chat), F, rtol=1e-14, atol=1e-15 * U[0])
    # S_L > 0: both states stream along +x with f close to 1 -> the left flux
    UL = np.array([1.0, 0.995, 0.0, 0.0])
    UR = np.array([0.7, 0.69, 0.01, 0.0])
    assert min(orc.wave_speeds(UL, 0, chat)[0], orc.wave_speeds(UR, 0, chat)[0]) > 0
    assert np.allclose(orc.hll(UL, UR, 0, chat), orc.flux(UL, 0, chat), rtol=1e-15, atol=0)
    # S_R < 0: mirror image -> the right flux
    UL2 = UR * np.array([1, -1, 1, 1])
    UR2 = UL * np.array([1, -1, 1, 1])
    assert np.allclose(orc.hll(UL2, UR2, 0, chat), orc.flux(UR2, 0, chat), rtol=1e-15, atol=0)


def test_hll_equals_intermediate_state_form():
    """With S_L <= 0 <= S_R, Eq. (hyperbolic:hllflux2) equals the intermediate-state flux of
    Eq. (hyperbolic:hllflux1) read with calligraphic F_L in its second bracket
    (calF = F - S U along characteristics)."""
    chat = 1.0
    states = _rand_states(400, 8, fmax=0.8)
    for a, b in zip(states[::2], states[1::2]):
        for d in range(3):
            l1a, l3a = orc.wave_speeds(a, d, chat)
            l1b, l3b = orc.wave_speeds(b, d, chat)
            SR, SL = max(l3a, l3b), min(l1a, l1b)
            if not (SL <= 0 <= SR):
                continue
            FL, FR = orc.flux(a, d, chat), orc.flux(b, d, chat)
            cL, cR = FL - SL * a, FR - SR * b
            star = 0.5 * (cL + cR) + 0.5 * (cL - cR) * (SR + SL) / (SR - SL)
            assert np.allclose(orc.hll(a, b, d, chat), star, rtol=1e-12, atol=1e-13)


def test_f_crit_is_where_closure_slope_is_singular():
    """f_crit = 2 sqrt(3)/5 (Section 4.3.6) is where 5 sqrt(4 - 3 f^2) - 8 = 0, i.e. where
    d(f chi)/df... in the paper's ODE the factor 5 s - 8 vanishes; check it against chi."""
    fc = GOLD["f_crit"]["value"]
    assert fc == pytest.approx(2 * math.sqrt(3) / 5, rel=1e-15)
    s = math.sqrt(4 - 3 * fc * fc)
    assert 5 * s - 8 == pytest.approx(0.0, abs=1e-14)
    # d(chi)/df via the oracle, equals 2 f / s (chi = (5 - 2 s)/3); at f_crit: 2 f_crit / (8/5)
    h = 1e-6
    dchi = (orc.chi(fc + h) - orc.chi(fc - h)) / (2 * h)
    assert dchi == pytest.approx(2 * fc / s, rel=1e-8)
