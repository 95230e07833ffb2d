"""GPU: failures are reported as statuses and leave the context usable (no device fault, trap or hang
is ever provoked; every failure here comes from the inputs or a host-side limit)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

from split_bounds import split_bound

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_nonfinite_input_reported_then_recovers(rhd, precision):
    case = wl.parity_case("nan", (20, 12, 10), bc="periodic", exchange="full", n_sub=2, seed=41, precision=precision)
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    f = case["fields"]
    E = f["E"].copy()
    E[5, 6, 7] = np.nan
    g.set_moments(E, f["Fx"], f["Fy"], f["Fz"])
    g.radiation_subcycle(2, case["chat"], case["dt"])
    with pytest.raises(rhd.RhdError) as ei:
        g.get_stats()
    assert ei.value.status == rhd.ERR_NONFINITE
    assert g.get_stats(allow_nonfinite=True)["n_nonfinite"] > 0
    # the context is still usable: a fresh finite state (moments and gas, whose T the exchange
    # with the NaN cell may have spoiled) advances cleanly
    g.reset_stats()
    g.load_case(case)
    g.radiation_subcycle(2, case["chat"], case["dt"])
    st = g.get_stats()
    assert st["n_nonfinite"] == 0 and np.isfinite(st["sum_E"])
    g.close()


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_superluminal_input_is_rescaled(rhd, precision):
    """|F| > cE on input is outside the realizable set: the closure clamps f and the update rescales
    the flux (Section 2.2); the result follows the oracle, which does the same."""
    case = wl.parity_case("flux", (16, 12, 10), bc="periodic", exchange="equilibrium", n_sub=1, seed=42,
                          precision=precision)
    f = case["fields"]
    f["Fx"] = f["Fx"].copy()
    f["Fx"][3, 4, 5] = 5.0 * case["desc"]["c"] * f["E"][3, 4, 5]  # |F| = 5 cE
    ref, st_ref = orc.subcycles(case)
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(1, case["chat"], case["dt"])
    st = g.get_stats()
    out = g.get_moments()
    g.close()
    assert st["n_realizability_fix"] > 0 and st_ref["n_realizability_fix"] > 0 and st["n_nonfinite"] == 0
    tol = split_bound(case, 1) if precision == "split" else FP64_TOL
    sE = float(np.max(np.abs(ref["E"])))
    assert float(np.max(np.abs(out["E"] - ref["E"]))) <= tol * sE
    for k in ("Fx", "Fy", "Fz"):
        assert float(np.max(np.abs(out[k] - ref[k]))) <= tol * case["desc"]["c"] * sE, k
    if precision == "fp64":
        assert st["n_realizability_fix"] == st_ref["n_realizability_fix"]
    F = np.sqrt(out["Fx"] ** 2 + out["Fy"] ** 2 + out["Fz"] ** 2)
    assert np.all(F <= case["desc"]["c"] * out["E"] * (1 + 1e-6))


def test_step_arguments_rejected_context_usable(rhd):
    case = wl.parity_case("args", (16, 8, 8), n_sub=1, seed=43, precision="split")
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    c, dt = case["chat"], case["dt"]
    dx = min(case["desc"]["dx"])
    for bad, status in (((c, 2 * case["desc"]["cfl"] * dx / c), rhd.ERR_CFL), ((0.0, dt), rhd.ERR_ARG),
                        ((-1.0, dt), rhd.ERR_ARG), ((2.0 * case["desc"]["c"], dt), rhd.ERR_CFL),
                        ((c, float("nan")), rhd.ERR_ARG)):
        with pytest.raises(rhd.RhdError) as ei:
            g.radiation_subcycle(1, *bad)
        assert ei.value.status == status, bad
    with pytest.raises(rhd.RhdError) as ei:
        g.radiation_subcycle(-1, c, dt)
    assert ei.value.status == rhd.ERR_ARG
    g.radiation_subcycle(1, c, dt)
    assert g.get_stats()["n_subcycles"] == 1
    g.close()


def test_forced_out_of_memory_then_recovers(rhd, monkeypatch):
    case = wl.parity_case("oom", (48, 32, 32), n_sub=1, seed=44, precision="split")
    monkeypatch.setenv("RHD_DEVICE_MEMORY_LIMIT", str(1 << 20))
    with pytest.raises(rhd.RhdError) as ei:
        rhd.Grid(case["desc"])
    assert ei.value.status == rhd.ERR_OOM
    # without the limit the same process creates and steps the grid
    monkeypatch.delenv("RHD_DEVICE_MEMORY_LIMIT")
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(1, case["chat"], case["dt"])
    assert g.get_stats()["n_nonfinite"] == 0
    g.close()


def test_state_required_before_stepping(rhd):
    case = wl.parity_case("state", (16, 8, 8), n_sub=1, seed=45, precision="split")
    g = rhd.Grid(case["desc"])
    with pytest.raises(rhd.RhdError) as ei:
        g.radiation_subcycle(1, case["chat"], case["dt"])
    assert ei.value.status == rhd.ERR_STATE
    with pytest.raises(rhd.RhdError) as ei:
        g.get_moments()
    assert ei.value.status == rhd.ERR_STATE
    g.close()


def test_subnormal_energy_floor_rejected(rhd):
    """E_floor must be a normal number of the arithmetic that divides by E: FP64 everywhere, FP32 on
    split grids (whose closure takes FP32 reciprocals of E); a subnormal floor is an argument error."""
    case = wl.parity_case("floor", (8, 6, 5), bc="periodic", n_sub=1, seed=3, precision="split")
    for precision, floor in (("split", 1e-39), ("fp64", 1e-310)):
        with pytest.raises(rhd.RhdError) as ei:
            rhd.Grid(dict(case["desc"], precision=precision, E_floor=floor))
        assert ei.value.status == rhd.ERR_ARG
    g = rhd.Grid(dict(case["desc"], precision="split", E_floor=2e-38))  # normal in FP32: accepted
    g.close()


def test_tma_wait_timeout_is_reported_and_the_context_recovers(rhd):
    """The bounded wait of the two-pass corrector's TMA staging, made to run out on the host's order
    (rhd_set_wait_limit(0): every plane wait gives up at once; the copy in flight is still awaited with
    the full bound before each block exits).  The timed-out tiles keep no new values, rhd_get_stats
    reports RHD_ERR_TIMEOUT with the count, and the same context, with the state reloaded and the
    default limit, steps to the oracle's result."""
    import ctypes

    case = wl.parity_case("timeout", (37, 11, 9), bc="outflow", exchange="full", beta_tau=True, n_sub=2, seed=23,
                          precision="split")
    g = rhd.Grid(case["desc"])
    try:
        g.set_launch_config(dict(variant="twopass", tile=(32, 8), z_chunk=4, staging="tma"))
    except rhd.RhdError:
        g.close()
        pytest.skip("TMA staging unavailable (no tensor-map encoder in the driver)")
    g.load_case(case)
    g.set_wait_limit(0)
    g.radiation_subcycle(1, case["chat"], case["dt"])
    s = rhd.Stats()
    status = rhd.lib().rhd_get_stats(g._ctx, ctypes.byref(s))
    assert status == rhd.ERR_TIMEOUT
    # one timed-out tile per (tile, z chunk) block: 2 x 2 tiles in x, y and 3 chunks of 4 planes
    assert s.as_dict()["wait_timeouts"] == 2 * 2 * 3
    # recovery in the same context: reload the state, restore the limit, clear the counters, step again
    g.set_wait_limit(-1)
    g.reset_stats()
    g.load_case(case)
    g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    st = g.get_stats()
    g.close()
    assert st["wait_timeouts"] == 0 and st["n_nonfinite"] == 0
    ref, _ = orc.subcycles(case)
    sE = float(np.max(np.abs(ref["E"])))
    tol = split_bound(case, case["n_sub"])
    assert float(np.max(np.abs(out["E"] - ref["E"]))) <= tol * sE
    for k in ("Fx", "Fy", "Fz"):
        assert float(np.max(np.abs(out[k] - ref[k]))) <= tol * case["desc"]["c"] * sE, k
    assert float(np.max(np.abs(out["T"] - ref["T"]))) <= tol * float(np.max(ref["T"]))
