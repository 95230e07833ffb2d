"""CPU pins of the oracle's slope limiters (reading r4: componentwise on (E, G)), against the
definitions, and of the monotonized central (MC) limiter inside the scheme.

MC (van Leer 1977): slope = minmod(2 dl, 2 dr, (dl + dr)/2) for left / right differences dl, dr; so
it is the central difference (dl + dr)/2 where neither difference is more than three times the
other, twice the smaller difference beyond that ratio, and zero at an extremum (dl dr <= 0).
Minmod: the difference nearer zero, zero at an extremum.  None: (dl + dr)/2."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl


@pytest.mark.parametrize("dl,dr,mc,minmod", [
    (1.0, 1.0, 1.0, 1.0),       # linear data: the central difference
    (0.3, 0.3, 0.3, 0.3),
    (1.0, 2.0, 1.5, 1.0),       # ratio 2 (< 3): central
    (2.0, 1.0, 1.5, 1.0),
    (1.0, 3.0, 2.0, 1.0),       # ratio 3: central (2) = twice the smaller (2)
    (1.0, 4.0, 2.0, 1.0),       # ratio 4 (> 3): twice the smaller
    (5.0, 1.0, 2.0, 1.0),
    (-1.0, -7.0, -2.0, -1.0),   # negative slopes: odd symmetry
    (-2.0, -1.0, -1.5, -1.0),
    (1.0, -1.0, 0.0, 0.0),      # extremum
    (-0.5, 2.0, 0.0, 0.0),
    (0.0, 1.0, 0.0, 0.0),       # flat on one side
    (1.0, 0.0, 0.0, 0.0),
])
def test_limiters_against_their_definitions(dl, dr, mc, minmod):
    assert orc.limited_slope(dl, dr, "mc") == mc
    assert orc.limited_slope(dl, dr, "minmod") == minmod
    assert orc.limited_slope(dl, dr, "none") == 0.5 * (dl + dr)


def test_mc_is_the_three_argument_minmod_on_random_pairs():
    g = np.random.Generator(np.random.PCG64(4))
    for dl, dr in g.normal(size=(2000, 2)) * np.exp(g.normal(size=(2000, 1))):
        args = (2 * dl, 2 * dr, 0.5 * (dl + dr))
        ref = 0.0 if not (all(a > 0 for a in args) or all(a < 0 for a in args)) else \
            math.copysign(min(abs(a) for a in args), args[0])
        got = orc.limited_slope(dl, dr, "mc")
        assert got == pytest.approx(ref, rel=1e-15, abs=0.0), (dl, dr)
        assert orc.limited_slope(dr, dl, "mc") == got            # symmetric in the two sides
        assert orc.limited_slope(-dl, -dr, "mc") == -got         # odd


def test_mc_advection_of_a_square_pulse_makes_no_new_extrema():
    """A limited slope keeps the face values between the neighbouring cell values, so a streaming
    square pulse (f = 1, exact upwinding, Section 3.3) gains no new extrema with MC, while the
    unlimited central slope overshoots."""
    def run(limiter):
        N = 64
        chat = 1.0
        desc = wl.base_desc((N, 1, 1), (1.0 / N, 1.0, 1.0), bc="periodic", c=chat, exchange="equilibrium",
                            limiter=limiter, E_floor=1e-12)
        x = (np.arange(N) + 0.5) / N
        E = np.where((x > 0.25) & (x < 0.5), 2.0, 1.0)
        shp = (1, 1, N)
        f = {"E": E.reshape(shp), "Fx": (chat * E).reshape(shp), "Fy": np.zeros(shp), "Fz": np.zeros(shp),
             "T": np.ones(shp), "rho": np.ones(shp), "vx": None, "vy": None, "vz": None, "kP": None,
             "kF": None, "j": None}
        out, _ = orc.subcycles({"desc": desc, "fields": f, "chat": chat, "dt": 0.4 / N, "n_sub": 40})
        return out["E"][0, 0]
    E_mc = run("mc")
    assert E_mc.max() <= 2.0 + 1e-12 and E_mc.min() >= 1.0 - 1e-12
    assert E_mc.max() > 1.99                       # the plateau survives (MC is not over-diffusive)
    E_none = run("none")
    assert E_none.max() > 2.0 + 1e-3 or E_none.min() < 1.0 - 1e-3
