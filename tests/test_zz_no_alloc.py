"""The no-allocation entry point rhd_subcycle_noalloc, for callers that cannot call cudaMalloc (for
example code running while another component owns the device memory through its own pool), must
give the same result as the context-based entry point.  Two calls in a row share the library's
static scratch array; each is compared with rhd_radiation_subcycle at the FP64 tolerance.  This file
is collected last, so a failure here comes after every other test has run."""
import numpy as np
import pytest

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


def _noalloc(torch, rhd, case, n_sub):
    f = case["fields"]
    dev = {k: (None if f[k] is None else torch.from_numpy(np.ascontiguousarray(f[k])).cuda()) for k in f}
    outs = {k: torch.empty_like(dev["E"]) for k in ("E", "Fx", "Fy", "Fz", "T")}
    st = rhd.subcycle_noalloc(case["desc"], n_sub, case["chat"], case["dt"], dev["E"], dev["Fx"], dev["Fy"],
                              dev["Fz"], dev["rho"], dev["T"], outs["E"], outs["Fx"], outs["Fy"], outs["Fz"],
                              outs["T"], vx=dev["vx"], vy=dev["vy"], vz=dev["vz"], kP=dev["kP"], kF=dev["kF"],
                              j=dev["j"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in outs.items()}, st


def _check(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    assert np.max(np.abs(out["E"] - ref["E"])) <= FP64_TOL * sE
    for k in ("Fx", "Fy", "Fz"):
        assert np.max(np.abs(out[k] - ref[k])) <= FP64_TOL * desc["c"] * sE, k
    assert np.max(np.abs(out["T"] - ref["T"])) <= FP64_TOL * float(np.max(np.abs(ref["T"])))


def test_noalloc_matches_context_entry_point_two_calls(env):
    torch, rhd = env
    first = wl.parity_case("na1", (20, 13, 9), bc="periodic", exchange="full", beta_tau=True, n_sub=3, seed=71,
                           with_j=True)
    second = wl.parity_case("na2", (16, 16, 12), bc=(["outflow", "reflect", "periodic"], ["outflow", "reflect",
                            "periodic"]), exchange="absorb", n_sub=4, seed=72)
    for case in (first, second):
        ref = _reference(rhd, case, case["n_sub"])
        out, st = _noalloc(torch, rhd, case, case["n_sub"])
        _check(out, ref, case["desc"])
        assert st["n_subcycles"] == case["n_sub"] and st["n_nonfinite"] == 0


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, rhd = env
    n = rhd.NOALLOC_MAX_CELLS + 1
    desc = wl.base_desc((n, 1, 1), (1.0 / n, 1.0, 1.0))
    t = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(rhd.RhdError) as ei:
        rhd.subcycle_noalloc(desc, 1, 1.0, 0.1 / n, t, t, t, t, t, t, t, t, t, t, t)
    assert ei.value.status == rhd.ERR_ARG and "at most" in str(ei.value)
