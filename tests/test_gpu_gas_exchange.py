"""GPU: the paper's placement of the stiff exchange (Section 3.1 step 2, Section 3.4: S_i integrated once
per gas step), rhd_gas_exchange on grids with RHD_FLAG_EXCHANGE_ON_GAS_STEP, against the oracle
(oracle/gas.py gas_exchange) element by element, alone and inside whole cycles (exchange, gas step,
subcycles without exchange, source correction; tests/oracle_cycles.py run_cycles).

The exchange runs in FP64 on both precisions, so the cell-wise comparison holds the FP64 path's bound
(1e-12 normwise) on split grids too; whole cycles on split grids hold the split gas step's bound."""
import numpy as np
import pytest

from oracle import gas as ogas
from oracle_cycles import run_cycles
from paper_1306_0010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SPLIT_GAS_TOL = 1e-4  # the split gas step's bound (tests/test_gpu_gas.py)


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def exchange_case(precision, seed=3, kP_array=False, n=(12, 9, 7), K_hot=False):
    case = wl.gas_case("xchg", n, bc=(["periodic", "outflow", "reflect"], ["periodic", "reflect", "outflow"]),
                       exchange="full", kappa=5.0, kappa_rho_pow=1, seed=seed, precision=precision, kF_array=kP_array)
    if K_hot:  # radiation far below the gas's equilibrium value: a strong, stiff exchange
        f = case["fields"]
        case["fields"] = dict(f, E=0.05 * f["E"], Fx=0.05 * f["Fx"], Fy=0.05 * f["Fy"], Fz=0.05 * f["Fz"])
    return case


def errors(out_rad, out_T, ref_rad, ref_T, c):
    sE = float(np.max(np.abs(ref_rad["E"])))
    e = {"E": float(np.max(np.abs(out_rad["E"] - ref_rad["E"]))) / sE,
         "T": float(np.max(np.abs(out_T - ref_T))) / float(np.max(np.abs(ref_T)))}
    for k in ("Fx", "Fy", "Fz"):
        e[k] = float(np.max(np.abs(out_rad[k] - ref_rad[k]))) / (c * sE)
    return e


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("kP_array,K_hot,dt", [(False, False, 0.05), (True, False, 0.05), (False, True, 0.5),
                                               (False, True, 1e6)], ids=["law", "arrays", "stiff", "equilibrium"])
def test_exchange_once_per_gas_step_matches_the_oracle(rhd, precision, kP_array, K_hot, dt):
    case = exchange_case(precision, kP_array=kP_array, K_hot=K_hot)
    desc = dict(case["desc"], flags=rhd.FLAG_EXCHANGE_ON_GAS_STEP)
    g = rhd.Grid(desc)
    g.load_case(case)
    g.gas_exchange(dt, case["chat"])
    out = g.get_moments()
    T = g.get_gas_state()
    st = g.get_stats()
    g.close()
    f = case["fields"]
    gas = {k: f[k] for k in ("rho", "vx", "vy", "vz", "T")}
    gas["kP"] = f.get("kP")
    ref_gas, ref_rad, fb = ogas.gas_exchange(desc, gas, {k: f[k] for k in ("E", "Fx", "Fy", "Fz")}, dt, case["chat"])
    e = errors(out, T, ref_rad, ref_gas["T"], desc["c"])
    assert max(e.values()) <= FP64_TOL, e
    assert st["n_theta_fallback"] == fb and st["n_nonfinite"] == 0
    assert not np.allclose(T, f["T"])  # it did exchange


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("split", SPLIT_GAS_TOL)])
def test_whole_cycles_with_the_exchange_per_gas_step(rhd, precision, tol):
    """Three whole cycles with the exchange before each gas step and none in the subcycles, through
    Grid.gas_cycle, against the oracle's cycles of the same placement."""
    case = exchange_case(precision, seed=5, n=(12, 10, 8))
    case["chat"] = 2.0
    dt = case["dt_gas"]
    n_cyc = 3
    ref_gas, ref_rad, n = run_cycles(case, n_cyc * dt, exchange_on_gas_step=True, dt_fixed=dt)
    assert n == n_cyc
    desc = dict(case["desc"], flags=rhd.FLAG_EXCHANGE_ON_GAS_STEP)
    g = rhd.Grid(desc)
    g.load_case(case)
    for _ in range(n_cyc):
        g.gas_cycle(case["chat"], dt_gas=dt)
    out_gas = g.get_gas()
    out_rad = g.get_moments()
    st = g.get_stats()
    g.close()
    assert st["n_nonfinite"] == 0
    e = errors(out_rad, out_gas["T"], ref_rad, ref_gas["T"], desc["c"])
    e["rho"] = float(np.max(np.abs(out_gas["rho"] - ref_gas["rho"]))) / float(np.max(ref_gas["rho"]))
    assert max(e.values()) <= tol, e


def test_flag_requires_full_exchange_and_a_single_grid(rhd):
    case = exchange_case("fp64")
    with pytest.raises(rhd.RhdError) as ei:
        rhd.Grid(dict(case["desc"], exchange="absorb", flags=rhd.FLAG_EXCHANGE_ON_GAS_STEP))
    assert ei.value.status == rhd.ERR_ARG
    c5 = wl.config5(n_grids=1, sizes=(16,), n_sub=1, precision="fp64")[0]
    with pytest.raises(rhd.RhdError) as ei:
        rhd.Ensemble([dict(c5["desc"], flags=rhd.FLAG_EXCHANGE_ON_GAS_STEP)])
    assert ei.value.status == rhd.ERR_ARG
    g = rhd.Grid(case["desc"])  # no flag: the subcycles exchange, and a second exchange is refused
    g.load_case(case)
    with pytest.raises(rhd.RhdError) as ei:
        g.gas_exchange(0.01, case["chat"])
    assert ei.value.status == rhd.ERR_STATE
    g.close()
