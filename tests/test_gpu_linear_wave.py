"""RHD linear waves on the GPU (Section 4.3.1, the paper's main validation of the RSLA with gas coupling):
one acoustic eigenmode of the linearised system run through whole Section 3.1 cycles (rhd_gas_step,
rhd_radiation_subcycle, rhd_gas_correct; FP64 grid), its phase speed and damping rate measured from the
k = 2 pi Fourier amplitude of delta rho.

- At 64 cells the GPU run equals the oracle's run of the same cycles (test_dispersion.oracle_wave): the
  measured Z agree to 1e-6 (both are FP64; the perturbation is 1e-6 of the background, so rounding of
  the O(1) fields is ~1e-10 of the signal per step).
- At the paper's 512 cells the measured Z matches the dispersion relation: the oracle's run at this
  resolution is off by 1.4e-5 (phase speed) and 2.2e-3 (damping rate), converging at first order from
  32 cells; the bounds are 1e-4 and 1e-2."""
import math

import numpy as np
import pytest

from oracle import dispersion as dsp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def gpu_wave(rhd, N, P0, C, Ch, tau, periods=1.0):
    from test_dispersion import wave_desc

    st, Z = dsp.mode_state(N, P0, C, Ch, tau)
    g = rhd.Grid(wave_desc(N, P0, C, Ch, tau))
    z = np.zeros((1, 1, N))
    g.set_gas_state(st["rho"], st["T"], st["vx"], z, z)
    g.set_moments(st["E"], st["Fx"], z, z)
    dt_gas = 0.4 / N
    times, rows = [0.0], [st["rho"][0, 0] - 1.0]
    for s in range(int(round(periods / dt_gas))):
        _, n_sub = g.gas_cycle(Ch, dt_gas=dt_gas)
        times.append((s + 1) * dt_gas)
        rows.append(g.get_gas()["rho"][0, 0] - 1.0)
    stats = g.get_stats()
    g.close()
    assert n_sub == math.ceil(Ch * (1 - 1e-12))
    assert stats["gas_nonfinite"] == 0 and stats["gas_energy_floors"] == 0
    return Z, dsp.measured_Z(times, np.array(rows))


# (P_0, Chat, tau) points of the paper's sweep (C = 1e4): the gas-energy-dominated case with strong
# energy exchange (P_0 C tau = 10), both reduced speeds of light, the radiation-pressure-dominated
# cases P_0 = 1 and 10, an optically thin and an optically thick wave
SWEEP = [(1e-3, 10.0, 1.0), (1e-3, 100.0, 1.0), (1.0, 10.0, 1.0), (10.0, 10.0, 1.0), (1e-3, 10.0, 0.1),
         (1e-3, 10.0, 100.0)]


@pytest.mark.parametrize("P0,Ch,tau", SWEEP, ids=[f"P{p:g}_Ch{c:g}_tau{t:g}" for p, c, t in SWEEP])
def test_linear_wave_equals_the_oracle_run(rhd, P0, Ch, tau):
    from test_dispersion import oracle_wave

    Z, Zg = gpu_wave(rhd, 64, P0, 1e4, Ch, tau)
    _, Zo = oracle_wave(64, P0, 1e4, Ch, tau)
    assert abs(Zg - Zo) <= 1e-6, (Zg, Zo)


def test_linear_wave_at_the_papers_resolution(rhd):
    Z, Zg = gpu_wave(rhd, 512, 1e-3, 1e4, 10.0, 1.0)
    assert abs(Zg.real - Z.real) <= 1e-4 * Z.real, (Z, Zg)
    assert abs(Zg.imag - Z.imag) <= 1e-2 * abs(Z.imag), (Z, Zg)


@pytest.mark.parametrize("P0", [1.0, 10.0])
def test_linear_wave_phase_speed_radiation_pressure_dominated(rhd, P0):
    """P_0 = 1 and 10 (Chat = 10, tau = 1): the phase speed at 512 cells within 1e-4 of the relation (the
    oracle's run at 64 cells is off by 1.1e-4, converging at first order).  The damping rate is not
    compared: the relation's is about 1e-4 of the real part, below the first-order scheme's own
    dissipation at this resolution (about 5e-4)."""
    Z, Zg = gpu_wave(rhd, 512, P0, 1e4, 10.0, 1.0)
    assert abs(Zg.real - Z.real) <= 1e-4 * Z.real, (Z, Zg)
    assert Zg.imag < 0.0  # damped
