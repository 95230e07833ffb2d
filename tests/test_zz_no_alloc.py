"""The no-allocation entry point rhd_subcycle_noalloc, for callers that cannot call cudaMalloc (for
example code running while another component owns the device memory through its own pool, or an
application that must keep its device footprint fixed once the library is loaded).  It must give the
oracle's result at the FP64 tolerance, and the same result as the context-based entry point, on two
calls in a row that share the library's static scratch array; a call must leave the free device memory
unchanged; a non-finite result is reported even when no statistics are requested.  This file is
collected last, so a failure here comes after every other test has run."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1306_0010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build, rhd

    build.build()
    rhd.lib()
    return torch, rhd


def _reference(rhd, case, n_sub):
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(n_sub, case["chat"], case["dt"])
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    g.close()
    return out


def _device_inputs(torch, case):
    f = case["fields"]
    dev = {k: (None if f[k] is None else torch.from_numpy(np.ascontiguousarray(f[k])).cuda()) for k in f}
    outs = {k: torch.empty_like(dev["E"]) for k in ("E", "Fx", "Fy", "Fz", "T")}
    return dev, outs


def _call(rhd, case, n_sub, dev, outs, want_stats=True):
    return rhd.subcycle_noalloc(case["desc"], n_sub, case["chat"], case["dt"], dev["E"], dev["Fx"], dev["Fy"],
                                dev["Fz"], dev["rho"], dev["T"], outs["E"], outs["Fx"], outs["Fy"], outs["Fz"],
                                outs["T"], vx=dev["vx"], vy=dev["vy"], vz=dev["vz"], kP=dev["kP"], kF=dev["kF"],
                                j=dev["j"], want_stats=want_stats)


def _noalloc(torch, rhd, case, n_sub):
    dev, outs = _device_inputs(torch, case)
    st = _call(rhd, case, n_sub, dev, outs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in outs.items()}, st


def _check(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    assert np.max(np.abs(out["E"] - ref["E"])) <= FP64_TOL * sE
    for k in ("Fx", "Fy", "Fz"):
        assert np.max(np.abs(out[k] - ref[k])) <= FP64_TOL * desc["c"] * sE, k
    assert np.max(np.abs(out["T"] - ref["T"])) <= FP64_TOL * float(np.max(np.abs(ref["T"])))


def test_noalloc_matches_the_oracle_and_the_context_entry_point_two_calls(env):
    torch, rhd = env
    first = wl.parity_case("na1", (20, 13, 9), bc="periodic", exchange="full", beta_tau=True, n_sub=3, seed=71,
                           with_j=True)
    second = wl.parity_case("na2", (16, 16, 12), bc=(["outflow", "reflect", "periodic"], ["outflow", "reflect",
                            "periodic"]), exchange="absorb", n_sub=4, seed=72)
    for case in (first, second):
        out, st = _noalloc(torch, rhd, case, case["n_sub"])
        assert st["n_subcycles"] == case["n_sub"] and st["n_nonfinite"] == 0
        oracle_out, _ = orc.subcycles(case)
        _check(out, oracle_out, case["desc"])
        _check(out, _reference(rhd, case, case["n_sub"]), case["desc"])


def test_noalloc_leaves_free_device_memory_unchanged(env):
    """On a grid near the scratch limit: one warm-up call (module loading), then the free device memory
    before and after a second call is the same."""
    torch, rhd = env
    n = (128, 128, 60)
    assert n[0] * n[1] * n[2] <= rhd.NOALLOC_MAX_CELLS
    case = wl.parity_case("na_mem", n, bc="periodic", exchange="full", beta_tau=True, n_sub=2, seed=73)
    dev, outs = _device_inputs(torch, case)
    _call(rhd, case, 2, dev, outs)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _call(rhd, case, 2, dev, outs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_reports_nonfinite_results_without_stats(env):
    torch, rhd = env
    case = wl.parity_case("na_nan", (12, 10, 8), bc="periodic", exchange="full", n_sub=1, seed=74)
    case["fields"] = dict(case["fields"], E=case["fields"]["E"].copy())
    case["fields"]["E"][3, 4, 5] = np.nan
    dev, outs = _device_inputs(torch, case)
    with pytest.raises(rhd.RhdError) as ei:
        _call(rhd, case, 1, dev, outs, want_stats=False)
    assert ei.value.status == rhd.ERR_NONFINITE
    # the next call on clean inputs succeeds (the counters start at zero on every call)
    clean = wl.parity_case("na_nan", (12, 10, 8), bc="periodic", exchange="full", n_sub=1, seed=74)
    dev, outs = _device_inputs(torch, clean)
    assert _call(rhd, clean, 1, dev, outs)["n_nonfinite"] == 0


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, rhd = env
    n = rhd.NOALLOC_MAX_CELLS + 1
    desc = wl.base_desc((n, 1, 1), (1.0 / n, 1.0, 1.0))
    t = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(rhd.RhdError) as ei:
        rhd.subcycle_noalloc(desc, 1, 1.0, 0.1 / n, t, t, t, t, t, t, t, t, t, t, t)
    assert ei.value.status == rhd.ERR_ARG and "at most" in str(ei.value)
