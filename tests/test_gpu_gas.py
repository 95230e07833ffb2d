"""GPU parity of the gas step (Section 3.1 steps 3 and 6, Section 3.4) through the C ABI against the
NumPy oracle (oracle/gas.py), element by element.

Tolerance: the kernels and the oracle evaluate the same FP64 formulas; they differ only in rounding
(the kernels multiply by reciprocals of dx, gamma - 1 and mu/k_B, and the compiler contracts products
and sums into fused multiply-adds).  One step is a few hundred operations per cell, each off by at most
an ulp, and the branches of the Riemann solver and the limiter are continuous, so a flipped branch also
costs only rounding: normwise errors stay near 1e-15 (measured up to 6e-16).  The bound used is the FP64
path's, GAS_TOL = 1e-12 per field (rho by max rho, v by max(|v| + a), T by max T), also for a whole cycle
(gas step, radiation subcycles, correction).

Split grids compute the face fluxes, the sources, the half step W^{n+1/2} and the increments in FP32
(inputs truncated to FP32, hardware reciprocal and square root approximations) and add the increments
to the FP64 state.  A face flux carries a relative error of at most about 50 FP32 ulps (2^-24 each: the
truncated inputs and some 25 dependent operations), 3e-6 of the flux scale rho (|v| + a)^2; a step adds
the differences of 2 faces in each of 3 directions times dt/dx (below the Courant number, 1/2) in each
of two stages, and the flux scale is up to (|v| + a)^2 ~ 4 times the field scales above:
2 x 6 x 0.5 x 3e-6 x 4 = 7e-5.  The increments of v and T are formed from those of rho, M and E
without cancellation (k_gas.cu), each a few FP32 ulps of the increment itself, and W^{n+1/2} in FP32 is
within the truncation the FP32 fluxes apply to their inputs anyway.  The bound used is SPLIT_GAS_TOL =
1e-4."""
import math

import numpy as np
import pytest

from oracle import gas as ogas
from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAS_TOL = 1e-12
SPLIT_GAS_TOL = 1e-4


@pytest.fixture(scope="module")
def rhd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd as binding

    build.build()
    binding.lib()
    return binding


def gas_in(case):
    f = case["fields"]
    return {k: f.get(k) for k in ("rho", "vx", "vy", "vz", "T", "kF")}


def rad_in(fields):
    return {k: fields[k] for k in ("E", "Fx", "Fy", "Fz")}


def gas_errors(out, ref, desc):
    a = np.sqrt(desc["gamma"] * ref["T"] / desc["mu_over_kB"])
    vs = float(np.max(np.sqrt(ref["vx"] ** 2 + ref["vy"] ** 2 + ref["vz"] ** 2) + a))
    e = {"rho": float(np.max(np.abs(out["rho"] - ref["rho"]))) / float(np.max(ref["rho"])),
         "T": float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(ref["T"]))}
    for k in ("vx", "vy", "vz"):
        e[k] = float(np.max(np.abs(out[k] - ref[k]))) / vs
    return e


GAS_CASES = [
    dict(name="3d_periodic_bt_kF", n=(9, 7, 5), bc="periodic", kF_array=True),
    dict(name="3d_mixed_bc_mc", n=(12, 9, 7), limiter="mc",
         bc=(["outflow", "reflect", "dirichlet"], ["reflect", "dirichlet", "periodic"]),
         dirichlet=([[0.0] * 4, [0.0] * 4, [1.5, 0.2, 0.1, 2.0]], [[0.0] * 4, [1.1, 0.0, 0.3, 0.0], [0.0] * 4])),
    dict(name="3d_ragged_tiles", n=(37, 11, 6), bc="outflow", kappa_rho_pow=2, kappa=0.5),
    dict(name="3d_no_beta_tau_kpow0", n=(10, 8, 6), bc="reflect", beta_tau=False, kappa_rho_pow=0, kappa=3.0),
    dict(name="3d_split_grid", n=(10, 8, 6), bc="periodic", precision="split"),
    dict(name="3d_split_mixed_bc_kF", n=(19, 9, 7), precision="split", limiter="mc", kF_array=True,
         bc=(["reflect", "periodic", "outflow"], ["outflow", "periodic", "dirichlet"]),
         dirichlet=([[0.0] * 4] * 3, [[0.0] * 4, [0.0] * 4, [1.3, 0.0, 0.2, 0.5]])),
    dict(name="2d_split_reflect", n=(21, 10, 1), bc="reflect", precision="split"),
    dict(name="3d_gas_at_rest", n=(8, 6, 5), bc="outflow", with_v=False),
    dict(name="2d_reflect_periodic", n=(17, 13, 1), bc=(["reflect", "periodic", "periodic"],
                                                      ["reflect", "periodic", "periodic"])),
    dict(name="2d_outflow_unlimited", n=(11, 6, 1), bc="outflow", limiter="none"),
    dict(name="2d_dirichlet_kF", n=(9, 14, 1), bc=(["dirichlet", "outflow", "periodic"], ["outflow", "reflect", "periodic"]),
         dirichlet=([[2.0, 0.5, 0.0, 0.0], [0.0] * 4, [0.0] * 4], [[0.0] * 4] * 3), kF_array=True),
    dict(name="1d_outflow_none", n=(33, 1, 1), bc="outflow", limiter="none"),
    dict(name="1d_n3_reflect", n=(3, 1, 1), bc="reflect"),
]


@pytest.mark.parametrize("kw", GAS_CASES, ids=[c["name"] for c in GAS_CASES])
def test_gas_step_and_correction_match_oracle(rhd, kw):
    kw = dict(kw)
    name = kw.pop("name")
    case = wl.gas_case(name, seed=len(name), **kw)
    desc, dt = case["desc"], case["dt_gas"]
    tol = SPLIT_GAS_TOL if desc["precision"] == "split" else GAS_TOL
    g = rhd.Grid(desc)
    g.load_case(case)
    g.gas_step(dt)
    out1 = g.get_gas()
    ref1, pend, floors = ogas.gas_step(desc, gas_in(case), rad_in(case["fields"]), dt)
    e = gas_errors(out1, ref1, desc)
    assert max(e.values()) <= tol, ("step", e)
    # the radiation at t^{n+1}, then the correction
    r1 = case["rad1"]
    g.set_moments(r1["E"], r1["Fx"], r1["Fy"], r1["Fz"])
    g.gas_correct()
    out2 = g.get_gas()
    st = g.get_stats()
    g.close()
    ref2, floors2 = ogas.gas_correct(desc, ref1, pend, r1)
    e = gas_errors(out2, ref2, desc)
    assert max(e.values()) <= tol, ("correction", e)
    assert st["gas_nonfinite"] == 0
    assert st["gas_energy_floors"] == floors + floors2
    print(name, "max normwise error", max(e.values()))


@pytest.mark.parametrize("precision,tol", [("fp64", GAS_TOL), ("split", SPLIT_GAS_TOL)])
def test_whole_cycle_matches_oracle(rhd, precision, tol):
    """Section 3.1 steps 3-6: gas step, n_sub radiation subcycles with the new gas, source correction."""
    case = wl.gas_case("cycle", (12, 10, 8), bc=(["periodic", "outflow", "reflect"], ["periodic", "outflow", "outflow"]),
                       precision=precision, seed=41, n_sub=4, kF_array=True)
    desc = case["desc"]
    g = rhd.Grid(desc)
    g.load_case(case)
    dt_gas, n_sub = g.gas_cycle(case["chat"], dt_gas=case["dt_gas"])
    assert n_sub == 1  # dt_gas is far below the radiation Courant limit at chat = 1
    out = g.get_gas()
    mom = g.get_moments()
    g.close()
    ref1, pend, _ = ogas.gas_step(desc, gas_in(case), rad_in(case["fields"]), dt_gas)
    rcase = dict(case, fields=dict(case["fields"], rho=ref1["rho"], vx=ref1["vx"], vy=ref1["vy"], vz=ref1["vz"],
                                   T=ref1["T"]))
    rad, _ = orc.subcycles(rcase, n_sub=n_sub, chat=case["chat"], dt=dt_gas / n_sub)
    ref1 = dict(ref1, T=rad["T"])
    ref2, _ = ogas.gas_correct(desc, ref1, pend, rad)
    e = gas_errors(out, ref2, desc)
    assert max(e.values()) <= tol, e
    sE = float(np.max(np.abs(rad["E"])))
    assert float(np.max(np.abs(mom["E"] - rad["E"]))) <= tol * sE


def test_sod_shock_tube_on_the_gpu(rhd):
    """Sod's problem (no radiation coupling): the GPU run equals the oracle's run and the exact solution's
    L1 error is that of the oracle (first-order convergence at the discontinuities)."""
    n = 200
    desc = wl.base_desc((n, 1, 1), (1.0 / n, 1.0, 1.0), bc="outflow", gamma=1.4, c=100.0, kappa_F=0.0,
                        kappa_P=0.0, E_floor=1e-30)
    x = (np.arange(n) + 0.5) / n
    left = (x < 0.5).reshape(1, 1, n)
    rho = np.where(left, 1.0, 0.125)
    T = np.where(left, 1.0, 0.1) / rho
    z = np.zeros((1, 1, n))
    g = rhd.Grid(desc)
    g.set_gas_state(rho, T, z, z, z)
    E = np.full((1, 1, n), 1e-20)
    g.set_moments(E, z, z, z)
    dt = 0.001  # max signal speed 1.75: Courant number 0.35
    ref = {"rho": rho, "vx": z, "vy": z, "vz": z, "T": T}
    rad = {"E": E, "Fx": z, "Fy": z, "Fz": z}
    for _ in range(200):
        g.gas_step(dt)
        g.gas_correct()
        ref, pend, _ = ogas.gas_step(desc, ref, rad, dt)
        ref, _ = ogas.gas_correct(desc, ref, pend, rad)
    out = g.get_gas()
    g.close()
    e = gas_errors(out, ref, desc)
    assert max(e.values()) <= GAS_TOL, e
    assert float(np.mean(np.abs(out["rho"] - ref["rho"]))) < 1e-12
    # the exact solution's density plateaus: left state, post-shock region
    assert abs(float(out["rho"][0, 0, 10]) - 1.0) < 1e-12
    assert abs(float(out["rho"][0, 0, 160]) - 0.26557) < 2e-3


@pytest.fixture(scope="module")
def config4_full():
    return wl.config4(N=512, n_sub=1)


@pytest.mark.parametrize("precision,tol", [("split", SPLIT_GAS_TOL), ("fp64", GAS_TOL)])
def test_full_size_gas_step_sampled(rhd, config4_full, precision, tol):
    """The 512^3 throughput configuration (periodic): one gas step and its correction on the GPU; the
    oracle recomputes sampled 6^3 boxes (one at the periodic corner) and every element must match."""
    case = config4_full
    desc = dict(case["desc"], precision=precision)
    dt = 0.1 / 512
    g = rhd.Grid(desc)
    g.load_case(case)
    g.gas_step(dt)
    f = case["fields"]
    r1 = {"E": 1.1 * f["E"], "Fx": 0.9 * f["Fx"], "Fy": 0.9 * f["Fy"], "Fz": 0.9 * f["Fz"]}
    g.set_moments(r1["E"], r1["Fx"], r1["Fy"], r1["Fz"])
    g.gas_correct()
    out = g.get_gas()
    st = g.get_stats()
    g.close()
    assert st["gas_nonfinite"] == 0
    boxes = [((0, 0, 0), (6, 6, 6)), ((506, 506, 506), (512, 512, 512)), ((250, 31, 400), (256, 37, 406))]
    for lo, hi in boxes:
        ref, pend, _ = ogas.gas_step(desc, gas_in(case), rad_in(f), dt, box=(lo, hi))
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        ref, _ = ogas.gas_correct(desc, ref, pend, {k: v[sl] for k, v in r1.items()})
        e = gas_errors({k: v[sl] for k, v in out.items()}, ref, desc)
        assert max(e.values()) <= tol, (lo, e)


def test_gas_api_errors(rhd):
    case = wl.gas_case("errors", (6, 5, 4))
    g = rhd.Grid(case["desc"])
    with pytest.raises(rhd.RhdError) as ei:
        g.gas_step(0.01)  # no state yet
    assert ei.value.status == rhd.ERR_STATE
    g.load_case(case)
    with pytest.raises(rhd.RhdError) as ei:
        g.gas_correct()  # nothing pending
    assert ei.value.status == rhd.ERR_STATE
    for bad in (-1.0, math.inf, math.nan):
        with pytest.raises(rhd.RhdError) as ei:
            g.gas_step(bad)
        assert ei.value.status == rhd.ERR_ARG
    g.gas_step(0.0)
    g.gas_correct()
    out = g.get_gas()
    f = case["fields"]
    assert np.array_equal(out["rho"], f["rho"])  # a zero step changes nothing but rounding of v and T
    g.close()
    ens = rhd.Ensemble([case["desc"]])
    with pytest.raises(rhd.RhdError) as ei:
        rhd._check(ens._ctx, rhd.lib().rhd_gas_step(ens._ctx, 0.01))
    assert ei.value.status == rhd.ERR_STATE
    ens.close()


def test_checkpoint_after_gas_cycles_resumes_bitwise(rhd, tmp_path):
    case = wl.gas_case("ckpt", (10, 8, 6), precision="split", seed=77)
    a = rhd.Grid(case["desc"])
    a.load_case(case)
    for _ in range(2):
        a.gas_cycle(case["chat"], dt_gas=case["dt_gas"])
    path = str(tmp_path / "gas.npz")
    a.checkpoint(path)
    b = rhd.Grid.restore(path)
    for gr in (a, b):
        gr.gas_cycle(case["chat"], dt_gas=case["dt_gas"])
    ga, gb = a.get_gas(), b.get_gas()
    ma, mb = a.get_moments(), b.get_moments()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_config3_shell_coupled_cycles_reduced(rhd, precision):
    """The dusty shell of the 256^3 coupled benchmark at 40^3: two whole cycles of 25 radiation subcycles
    each (Delta t_gas = 25 radiation steps, gas Courant number 0.2) against the oracle's cycles
    (tests/oracle_cycles.py).  FP64: 1e-12.  Split: the gas bound per step for the gas, the derived
    radiation bound over the 50 subcycles for the moments."""
    from oracle_cycles import run_cycles
    from split_bounds import split_bound

    case = wl.config3(N=40, n_sub=25, precision=precision)
    dt_gas = 25 * case["dt"]
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    subs = [g.gas_cycle(case["chat"], dt_gas=dt_gas)[1] for _ in range(2)]
    out, mom, st = g.get_gas(), g.get_moments(), g.get_stats()
    g.close()
    assert subs == [25, 25]
    ref_gas, ref_rad, n = run_cycles(case, 2 * dt_gas, dt_fixed=dt_gas)
    assert n == 2
    if precision == "fp64":
        tol_gas = tol_rad = GAS_TOL
    else:
        tol_gas, tol_rad = 2 * SPLIT_GAS_TOL, split_bound(case, 50)
    e = gas_errors(out, ref_gas, case["desc"])
    assert max(e.values()) <= tol_gas, e
    sE = float(np.max(np.abs(ref_rad["E"])))
    er = {"E": float(np.max(np.abs(mom["E"] - ref_rad["E"]))) / sE}
    for k in ("Fx", "Fy", "Fz"):
        er[k] = float(np.max(np.abs(mom[k] - ref_rad[k]))) / (case["desc"]["c"] * sE)
    assert max(er.values()) <= tol_rad, er
    assert st["n_nonfinite"] == 0 and st["gas_nonfinite"] == 0
    print(precision, "config3 coupled 40^3: gas", max(e.values()), "radiation", max(er.values()))
