"""The oracle's reduced-speed-of-light helpers against closed forms (Sections 3.1, 3.2)."""
import math

import numpy as np
import pytest

from oracle import rsla


def uniform(n=(8, 6, 4), dx=(0.1, 0.2, 0.25), rho=2.0, T=3.0, E=5.0, kF=None, kappa=0.0, p=1, gamma=5.0 / 3.0,
            mu=1.0):
    shp = (n[2], n[1], n[0])
    desc = {"n": n, "dx": dx, "gamma": gamma, "mu_over_kB": mu, "kappa_F": kappa, "kappa_rho_pow": p}
    f = {"rho": np.full(shp, rho), "T": np.full(shp, T), "kF": None if kF is None else np.full(shp, kF)}
    return desc, f, np.full(shp, E)


def test_thin_limit_is_the_ideal_gas_sound_speed():
    # k_F = 0: no radiation pressure term; c_s^2 = gamma k_B T / mu for an ideal gas
    desc, f, E = uniform(kF=0.0, T=3.0, mu=0.5)
    c = rsla.effective_sound_speed(desc, f, E)
    assert np.allclose(c, math.sqrt((5.0 / 3.0) * 3.0 / 0.5), rtol=1e-15, atol=0)


def test_thick_limit_adds_the_radiation_pressure_with_index_four_thirds():
    # k_F dx >> 1: c^2 = (gamma P + Gamma_r P_r) / rho with P_r = E/3 and Gamma_r = 4/3
    desc, f, E = uniform(kF=600.0, rho=2.0, T=3.0, E=7.0)  # k_F dx_min = 60
    P, Pr = 2.0 * 3.0, 7.0 / 3.0
    c = rsla.effective_sound_speed(desc, f, E)
    assert np.allclose(c, math.sqrt(((5.0 / 3.0) * P + (4.0 / 3.0) * Pr) / 2.0), rtol=1e-15, atol=0)


def test_half_opacity_weight_at_ln2():
    # 1 - exp(-ln 2) = 1/2 exactly: the radiation term is half its thick value
    dxmin = 0.1
    desc, f, E = uniform(kF=math.log(2.0) / dxmin, rho=1.5, T=0.5, E=9.0)
    c = rsla.effective_sound_speed(desc, f, E)
    assert np.allclose(c, math.sqrt(((5.0 / 3.0) * 1.5 * 0.5 + 0.5 * (4.0 / 9.0) * 9.0) / 1.5), rtol=1e-14, atol=0)


def test_opacity_law_matches_array_and_speed_is_monotone_in_opacity():
    desc, f, E = uniform(kappa=3.0, p=2, rho=1.7)
    c_law = rsla.effective_sound_speed(desc, f, E)
    f2 = dict(f, kF=np.full_like(f["rho"], 3.0 * 1.7 * 1.7))
    assert np.array_equal(c_law, rsla.effective_sound_speed(desc, f2, E))
    speeds = [float(rsla.effective_sound_speed(desc, dict(f, kF=np.full_like(f["rho"], k)), E).max())
              for k in (0.0, 1.0, 10.0, 100.0, 1000.0)]
    assert all(a < b for a, b in zip(speeds, speeds[1:]))


def test_max_signal_speed_picks_the_fast_cell():
    desc, f, E = uniform(kF=0.0, T=1.0, mu=1.0)
    shp = f["rho"].shape
    f["vx"] = np.zeros(shp)
    f["vy"] = np.zeros(shp)
    f["vz"] = None
    f["vx"][2, 3, 4] = 3.0
    f["vy"][2, 3, 4] = -4.0  # |v| = 5
    assert rsla.max_signal_speed(desc, f, E) == pytest.approx(5.0 + math.sqrt(5.0 / 3.0), rel=1e-15)


def test_max_optical_depth_closed_form():
    # uniform k0 plus one hot cell: the longest axis (x: 8 x 0.25 = 2.0) through the hot cell
    desc, f, E = uniform(n=(8, 6, 4), dx=(0.25, 0.2, 0.1), kF=1.5)
    assert rsla.max_optical_depth(desc, f) == pytest.approx(1.5 * 2.0, rel=1e-15)
    f["kF"][1, 2, 3] = 11.5
    assert rsla.max_optical_depth(desc, f) == pytest.approx(1.5 * 2.0 + 10.0 * 0.25, rel=1e-15)
    # inactive directions do not count: a 1D row along y only
    desc1, f1, _ = uniform(n=(1, 6, 1), dx=(7.0, 0.2, 9.0), kF=2.0)
    assert rsla.max_optical_depth(desc1, f1) == pytest.approx(2.0 * 6 * 0.2, rel=1e-15)


def test_suggest_chat_cases():
    assert rsla.suggest_chat(100.0, 0.5, 0.3, 10.0) == 5.0       # optically thin: R v_max
    assert rsla.suggest_chat(100.0, 0.5, 4.0, 10.0) == 20.0      # diffusion: R v_max tau_max
    assert rsla.suggest_chat(10.0, 0.5, 4.0, 10.0) == 10.0       # capped at c


@pytest.mark.parametrize("v,chat", [(0.5, 4.0), (0.3, 7.0), (1e-3, 10.0), (0.7, 0.7), (2.0, 1.0)])
def test_time_steps_span_the_gas_step(v, chat):
    cfl, dx = 0.4, 1.0 / 96
    dt_gas, dt_rad, n = rsla.time_steps(cfl, dx, v, chat)
    dt_max = cfl * dx / chat
    assert dt_gas == cfl * dx / v
    assert dt_rad <= dt_max
    assert (n - 1) * dt_max < dt_gas                     # no fewer subcycles would do
    assert abs(n * dt_rad - dt_gas) <= 4 * n * np.spacing(dt_gas)
    if (v, chat) == (0.5, 4.0):
        assert n == 8 and dt_rad == dt_max                # chat / v_max = 8 exactly
