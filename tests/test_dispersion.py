"""RHD linear waves (Section 4.3.1): the dispersion relation of the linearised system against the
paper's quintic and the limits the paper (and Lowrie et al. 1999) give, and the coupled oracle (gas
step, radiation subcycles, energy exchange) propagating one acoustic eigenmode at the phase speed and
damping rate the dispersion relation predicts."""
import math

import numpy as np
import pytest

from oracle import gas as ogas
from oracle import oracle as orc
from oracle import dispersion as dsp
from paper_1306_0010_gb300 import workloads as wl

G = 5.0 / 3.0


def test_modes_are_the_roots_of_the_quintic():
    """The eigenvalues of the linearised system equal the roots of Eq. radlinearwave:ivp:dispersion
    (Newton-polished from each eigenvalue, the paper's solver) up to the terms of order P_0 tau / C the
    quintic leaves out."""
    r = np.random.default_rng(3)
    for _ in range(40):
        P0 = 10 ** r.uniform(-3, 1)
        C = 10 ** r.uniform(3, 4)
        Ch = 10 ** r.uniform(1, math.log10(C))
        tau = 10 ** r.uniform(-1, 2)
        Z, _ = dsp.linear_modes(P0, C, Ch, tau)
        q = dsp.ivp_quintic(P0, C, Ch, tau)
        for z in Z:
            root = dsp.newton_root(q, z)
            assert abs(np.polyval(q, root)) <= 1e-9 * np.max(np.abs(q)) * max(1.0, abs(root)) ** 5
            assert abs(root - z) <= 1e-5 * max(1.0, abs(z)) + 2 * P0 * tau / C, (P0, C, Ch, tau, z, root)


def test_printed_last_bracket_would_leave_the_radiation_acoustic_mode_unaffected_by_the_rsla():
    """The reading of the quintic's last bracket (Chat): with C as printed, the acoustic mode of a
    radiation-dominated optically thick medium would travel at a_0* for Chat = 10 << C, contrary to the
    paper's statement that this mode is always affected by the RSLA; the linearised equations give the
    reduced speed, and so does the quintic with Chat."""
    P0, C, Ch, tau = 10.0, 1e4, 10.0, 100.0
    a_star = dsp.radiation_acoustic_speed(P0)
    printed = np.roots(dsp.ivp_quintic(P0, C, Ch, tau, last_bracket=C))
    assert any(abs(z.real - a_star) < 0.05 * a_star and z.real > 0 for z in printed)
    Zm, _ = dsp.acoustic_mode(P0, C, Ch, tau)
    assert Zm.real < 0.8 < a_star
    reading = np.roots(dsp.ivp_quintic(P0, C, Ch, tau))
    assert min(abs(reading - Zm)) < 1e-3


def test_decoupled_limits():
    # no radiation energy (P_0 -> 0): the entropy mode Z = 0, adiabatic sound +-1 and the radiation pair
    Z, X = dsp.linear_modes(1e-12, 1e4, 30.0, 1e-9)
    want = sorted([-30.0 / math.sqrt(3.0), -1.0, 0.0, 1.0, 30.0 / math.sqrt(3.0)])
    assert np.allclose(Z.real, want, atol=1e-6)
    assert np.all(np.abs(Z.imag) < 1e-6)
    # each eigenvector solves the linear system
    A, B = dsp._matrices(0.3, 1e4, 30.0, 2.0, G)
    Z, X = dsp.linear_modes(0.3, 1e4, 30.0, 2.0)
    for j in range(5):
        w = 2 * math.pi * Z[j]
        assert np.linalg.norm((A - 1j * w * B) @ X[:, j]) < 1e-10 * np.linalg.norm(A)


@pytest.mark.parametrize("tau", [1e-3, 3e-3])
def test_optically_thin_damping(tau):
    """Eq. radlinearwave:acoustic:thin: z = 1 + i (gamma-1)^2 P_0 C tau / pi for the driven wave; for weak
    damping the temporal rate is the same, Z = 1 - i (gamma-1)^2 P_0 C tau / pi."""
    P0, C = 1e-3, 1e4
    Z, _ = dsp.acoustic_mode(P0, C, 100.0, tau)
    damp = (G - 1) ** 2 * P0 * C * tau / math.pi
    assert abs(Z.real - 1.0) < 2e-3
    assert Z.imag == pytest.approx(-damp, rel=0.01)


@pytest.mark.parametrize("P0", [0.1, 1.0, 10.0])
def test_optically_thick_speed_is_the_radiation_modified_sound_speed(P0):
    """Chat = C, tau >> max(1, P_0 C): the acoustic mode travels at a_0* of
    Eq. radlinearwave:radiationacousticspeed (Lowrie et al. 1999, their Eq. 45)."""
    Z, _ = dsp.acoustic_mode(P0, 1e3, 1e3, 1e4)
    assert Z.real == pytest.approx(dsp.radiation_acoustic_speed(P0), rel=0.01)


# ----------------------------------------------------------------------------- the coupled scheme

def wave_desc(N, P0, C, Ch, tau):
    return wl.base_desc((N, 1, 1), (1.0 / N, 1.0, 1.0), bc="periodic", c=C, a_rad=P0, gamma=G, mu_over_kB=G,
                        exchange="full", beta_tau=True, limiter="none", closure="p1", speeds="fixed", kappa_P=tau,
                        kappa_F=tau, kappa_rho_pow=1, theta_F=1.0, theta_E=1.0, E_floor=1e-30, cfl=0.4)


def oracle_wave(N, P0, C, Ch, tau, periods=1.0):
    """The oracle's Section 3.1 cycle (gas step, subcycles over dt_gas = 0.4 dx / a_0, correction) on
    one acoustic eigenmode; returns (predicted Z, measured Z)."""
    st, Z = dsp.mode_state(N, P0, C, Ch, tau)
    desc = wave_desc(N, P0, C, Ch, tau)
    z = np.zeros((1, 1, N))
    gas = {"rho": st["rho"], "vx": st["vx"], "vy": z, "vz": z, "T": st["T"]}
    rad = {"E": st["E"], "Fx": st["Fx"], "Fy": z, "Fz": z}
    dt_gas = 0.4 / N
    n_sub = math.ceil(dt_gas / (0.4 / N / Ch) * (1 - 1e-12))
    times, rows = [0.0], [gas["rho"][0, 0] - 1.0]
    for s in range(int(round(periods / dt_gas))):
        g1, pend, _ = ogas.gas_step(desc, gas, rad, dt_gas)
        f = dict(rad, T=g1["T"], rho=g1["rho"], vx=g1["vx"], vy=g1["vy"], vz=g1["vz"], kP=None, kF=None, j=None)
        r1, _ = orc.subcycles({"desc": desc, "fields": f, "chat": Ch, "dt": dt_gas / n_sub, "n_sub": n_sub})
        rad = {k: r1[k] for k in ("E", "Fx", "Fy", "Fz")}
        gas, _ = ogas.gas_correct(desc, dict(g1, T=r1["T"]), pend, rad)
        times.append((s + 1) * dt_gas)
        rows.append(gas["rho"][0, 0] - 1.0)
    return Z, dsp.measured_Z(times, np.array(rows))


def test_oracle_propagates_the_acoustic_mode_at_the_predicted_speed_and_damping():
    """P_0 = 1e-3, C = 1e4, Chat = 10, tau = 1 (energy exchange strong, P_0 C tau = 10: the wave is nearly
    isothermal, Z = 0.7766 - 0.0305 i): one wave period on 32 and 64 cells."""
    errs = []
    for N in (32, 64):
        Z, Zm = oracle_wave(N, 1e-3, 1e4, 10.0, 1.0)
        errs.append((abs(Zm.real - Z.real) / Z.real, abs(Zm.imag - Z.imag) / abs(Z.imag)))
    assert errs[0][0] < 1e-3 and errs[0][1] < 0.12, errs
    assert errs[1][0] < 5e-4 and errs[1][1] < 0.05, errs
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1], errs


def test_rsla_criterion_keeps_the_acoustic_mode():
    """Gas-dominated case (P_0 = 1e-3, C = 1e4): while Chat >= tau (the static-diffusion criterion,
    Eq. rsla:staticdiffreq, at rest) the acoustic mode with the reduced speed stays within a few per
    cent of the mode with chat = c; well beyond it (tau = 10 Chat) its speed and damping change where the
    energy exchange still matters (Chat = 10, 100: tau ~ P_0 C).  The paper notes the criterion is
    sufficient, not necessary: at Chat = 1000, tau = 10^4 >> P_0 C the mode is adiabatic either way."""
    P0, C = 1e-3, 1e4
    for Ch in (10.0, 100.0, 1000.0):
        for tau in np.logspace(-2, math.log10(Ch), 12):
            Za, _ = dsp.acoustic_mode(P0, C, Ch, tau)
            Zc, _ = dsp.acoustic_mode(P0, C, C, tau)
            assert abs(Za - Zc) <= 0.06 * abs(Zc), (Ch, tau, Za, Zc)
    for Ch in (10.0, 100.0):
        Za, _ = dsp.acoustic_mode(P0, C, Ch, 10 * Ch)
        Zc, _ = dsp.acoustic_mode(P0, C, C, 10 * Ch)
        assert abs(Za.real - Zc.real) > 0.05 * Zc.real and abs(Za.imag) < 0.7 * abs(Zc.imag), (Ch, Za, Zc)


def test_oracle_acoustic_speed_in_the_radiation_dominated_case_is_the_reduced_one():
    """P_0 = 10, C = 1e4, Chat = 10, tau = 10: with chat = c the acoustic mode would travel at
    a_0* = 2.31 a_0; with the reduced speed the dispersion relation gives 0.775 a_0 (radiation pressure no
    longer supports the wave), and the oracle's coupled cycles travel at that speed.  The mode's own
    damping (1e-3) is below the scheme's at 32 cells, whose error is first order in the cell size (the
    gas / radiation splitting of Sec. 3.1 is formally first order)."""
    Z, Zm = oracle_wave(32, 10.0, 1e4, 10.0, 10.0)
    assert abs(Zm.real - Z.real) <= 3e-4 * Z.real, (Z, Zm)
    assert abs(Zm.real - dsp.radiation_acoustic_speed(10.0)) > 1.0
    assert -0.02 < Zm.imag < 0.0
