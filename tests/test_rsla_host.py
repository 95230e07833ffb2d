"""The library's host-side reduced-speed-of-light helpers (rhd_suggest_chat, rhd_time_steps: plain
host arithmetic, no GPU needed) against the oracle."""
import pytest

from oracle import rsla


def test_library_host_helpers_match_the_oracle():
    rhd = pytest.importorskip("paper_1306_0010_gb300.rhd")
    try:
        rhd.lib()
    except RuntimeError:
        pytest.skip("library not built")
    for args in [(100.0, 0.5, 0.3, 10.0), (100.0, 0.5, 4.0, 10.0), (10.0, 0.5, 4.0, 10.0), (3e5, 12.0, 25.0, 30.0)]:
        assert rhd.suggest_chat(*args) == rsla.suggest_chat(*args)
    for v, chat in [(0.5, 4.0), (0.3, 7.0), (1e-3, 10.0), (0.7, 0.7), (2.0, 1.0)]:
        assert rhd.time_steps(0.4, 1.0 / 96, v, chat) == rsla.time_steps(0.4, 1.0 / 96, v, chat)
    for bad in [(0.0, 0.5, 1.0, 10.0), (10.0, -1.0, 1.0, 10.0), (10.0, 0.5, -1.0, 10.0), (10.0, 0.5, 1.0, float("nan"))]:
        with pytest.raises(rhd.RhdError) as ei:
            rhd.suggest_chat(*bad)
        assert ei.value.status == rhd.ERR_ARG
    with pytest.raises(rhd.RhdError):
        rhd.time_steps(0.4, 0.0, 1.0, 1.0)
    # the subcycles spanning a given gas step: those of rhd_time_steps for its own dt_gas, and in
    # general the fewest of length <= cfl dx / chat
    for v, chat in [(0.5, 4.0), (0.3, 7.0), (0.7, 0.7)]:
        dg, dr, n = rsla.time_steps(0.4, 1.0 / 96, v, chat)
        assert rhd.subcycle_steps(0.4, 1.0 / 96, chat, dg) == (dr, n)
    for dg in (1e-3, 0.0125, 0.05, 0.3):
        dr, n = rhd.subcycle_steps(0.4, 1.0 / 80, 2.0, dg)
        assert dr == dg / n and dr <= 0.4 / 80 / 2.0 and (n == 1 or dg / (n - 1) > 0.4 / 80 / 2.0)
    with pytest.raises(rhd.RhdError):
        rhd.subcycle_steps(0.4, 1.0 / 80, 2.0, -1.0)
