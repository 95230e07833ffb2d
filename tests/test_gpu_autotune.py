"""GPU: the autotuner and explicit launch configurations.

Tuning times candidate launch configurations on the live state; it must leave the state (E, F,
T) and the statistics exactly as they were, keep the fastest candidate it measured, and every
candidate it offers must give results within the bound of its precision against the oracle."""
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


def errors(out, ref, desc):
    sE = float(np.max(np.abs(ref["E"])))
    e = {"E": float(np.max(np.abs(out["E"] - ref["E"]))) / sE}
    for k in ("Fx", "Fy", "Fz"):
        e[k] = float(np.max(np.abs(out[k] - ref[k]))) / (desc["c"] * sE)
    if desc["exchange"] == "full":
        e["T"] = float(np.max(np.abs(out["T"] - ref["T"]))) / float(np.max(np.abs(ref["T"])))
    return e


def snapshot(g):
    out = g.get_moments()
    out["T"] = g.get_gas_state()
    return out


def case_split():
    return wl.parity_case("tune_split", (40, 24, 36), bc=(["periodic", "outflow", "reflect"],
                                                           ["periodic", "outflow", "outflow"]),
                          exchange="full", beta_tau=True, with_j=True, n_sub=3, seed=31, precision="split")


def test_autotune_keeps_state_and_picks_fastest(rhd):
    case = case_split()
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(1, case["chat"], case["dt"])  # some statistics to preserve
    before, st_before = snapshot(g), g.get_stats()
    chosen, table = g.autotune(case["chat"], case["dt"], reps=2)
    after, st_after = snapshot(g), g.get_stats()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert st_before == st_after
    assert {c["variant"] for c in table} == {"fused", "twopass"}
    timed = [c for c in table if c["ms_per_subcycle"] >= 0]
    assert len(timed) == len(table)
    best = min(timed, key=lambda c: c["ms_per_subcycle"])
    assert (chosen["variant"], chosen["tile"], chosen["z_chunk"], chosen["staging"]) == \
        (best["variant"], best["tile"], best["z_chunk"], best["staging"])
    cur = g.launch_config()
    assert cur["ms_per_subcycle"] == best["ms_per_subcycle"]
    g.close()


def test_every_split_candidate_within_bound(rhd):
    case = case_split()
    ref, _ = orc.subcycles(case)
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    _, table = g.autotune(case["chat"], case["dt"], reps=1)
    g.close()
    assert len(table) >= 6
    for cfg in table:
        g = rhd.Grid(case["desc"])
        g.set_launch_config(cfg)
        got = g.launch_config()
        assert (got["variant"], got["tile"], got["z_chunk"], got["staging"]) == \
            (cfg["variant"], cfg["tile"], cfg["z_chunk"], cfg["staging"])
        g.load_case(case)
        g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
        out = snapshot(g)
        assert g.get_stats()["n_nonfinite"] == 0
        g.close()
        e = errors(out, ref, case["desc"])
        assert max(e.values()) <= split_bound(case, case["n_sub"]), (cfg, e)


def test_fp64_tuned_parity(rhd):
    case = wl.parity_case("tune_fp64", (24, 16, 40), bc="periodic", exchange="full", beta_tau=True, n_sub=3,
                          seed=32)
    ref, _ = orc.subcycles(case)
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    chosen, table = g.autotune(case["chat"], case["dt"], reps=2)
    assert chosen["variant"] == "fused" and chosen["tile"] == (16, 16)
    assert sorted({c["z_chunk"] for c in table}) == [8, 16, 32, 40]
    g.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    e = errors(snapshot(g), ref, case["desc"])
    g.close()
    assert max(e.values()) <= FP64_TOL, e


def test_flag_autotune_on_first_call_and_reuse(rhd):
    case = wl.parity_case("tune_flag", (36, 20, 18), bc="outflow", exchange="absorb", n_sub=2, seed=33,
                          precision="split")
    ref, _ = orc.subcycles(case)
    desc = dict(case["desc"], flags=rhd.FLAG_AUTOTUNE)
    g1 = rhd.Grid(desc)
    g1.load_case(case)
    assert g1.launch_config()["ms_per_subcycle"] < 0
    g1.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    c1 = g1.launch_config()
    assert c1["ms_per_subcycle"] >= 0
    e = errors(snapshot(g1), ref, case["desc"])
    assert max(e.values()) <= split_bound(case, case["n_sub"]), e
    g1.close()
    g2 = rhd.Grid(desc)  # same shape and mode: the first context's choice is reused
    g2.load_case(case)
    g2.radiation_subcycle(case["n_sub"], case["chat"], case["dt"])
    c2 = g2.launch_config()
    assert c2 == c1
    e = errors(snapshot(g2), ref, case["desc"])
    assert max(e.values()) <= split_bound(case, case["n_sub"]), e
    g2.close()


def test_ensemble_autotune(rhd):
    cases = [wl.config5(n_grids=1, sizes=(n,), n_sub=2, precision="fp64", seed_offset=70 + i)[0]
             for i, n in enumerate((16, 24, 32))]
    ens = rhd.Ensemble([c["desc"] for c in cases])
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    before = [(ens.get_moments(i), ens.get_gas_state(i)) for i in range(3)]
    chosen, table = ens.autotune(1.0, [c["dt"] for c in cases], reps=2)
    assert len(table) >= 3 and all(c["ms_per_subcycle"] >= 0 for c in table)
    assert chosen["z_chunk"] == min(table, key=lambda c: c["ms_per_subcycle"])["z_chunk"]
    for i in range(3):
        m, T = ens.get_moments(i), ens.get_gas_state(i)
        assert np.array_equal(T, before[i][1])
        for k in m:
            assert np.array_equal(m[k], before[i][0][k]), (i, k)
    ens.subcycle(2, 1.0, [c["dt"] for c in cases])
    for i, c in enumerate(cases):
        out = ens.get_moments(i)
        out["T"] = ens.get_gas_state(i)
        ref, _ = orc.subcycles(c, n_sub=2)
        assert max(errors(out, ref, c["desc"]).values()) <= FP64_TOL, i
    ens.close()


def test_ensemble_split_autotune_variants(rhd):
    cases = [wl.config5(n_grids=1, sizes=(n,), n_sub=2, precision="split", seed_offset=80 + i)[0]
             for i, n in enumerate((32, 48))]
    ens = rhd.Ensemble([c["desc"] for c in cases])
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    before = [(ens.get_moments(i), ens.get_gas_state(i)) for i in range(2)]
    chosen, table = ens.autotune(1.0, [c["dt"] for c in cases], reps=2)
    assert {c["variant"] for c in table} == {"fused", "twopass"}
    best = min(table, key=lambda c: c["ms_per_subcycle"])
    assert (chosen["variant"], chosen["z_chunk"]) == (best["variant"], best["z_chunk"])
    assert ens.launch_config()["variant"] == best["variant"]
    for i in range(2):
        m, T = ens.get_moments(i), ens.get_gas_state(i)
        assert np.array_equal(T, before[i][1])
        for k in m:
            assert np.array_equal(m[k], before[i][0][k]), (i, k)
    ens.subcycle(2, 1.0, [c["dt"] for c in cases])
    for i, c in enumerate(cases):
        out = ens.get_moments(i)
        out["T"] = ens.get_gas_state(i)
        ref, _ = orc.subcycles(c, n_sub=2)
        assert max(errors(out, ref, c["desc"]).values()) <= split_bound(c, 2), i
    ens.close()


def test_unsupported_launch_config_rejected(rhd):
    case = wl.parity_case("tune_bad", (16, 16, 16), n_sub=1, seed=34)  # FP64
    g = rhd.Grid(case["desc"])
    for cfg in (dict(variant="twopass", tile=(32, 8), z_chunk=16, staging="cpasync"),
                dict(variant="fused", tile=(32, 16), z_chunk=16, staging="cpasync"),
                dict(variant="fused", tile=(16, 8), z_chunk=16, staging="cpasync"),
                dict(variant="fused", tile=(16, 16), z_chunk=0, staging="cpasync"),
                dict(variant="fused", tile=(16, 16), z_chunk=8, staging="tma")):
        with pytest.raises(rhd.RhdError) as ei:
            g.set_launch_config(cfg)
        assert ei.value.status == rhd.ERR_ARG
    g.close()


def test_kernel_timer_counts_and_bytes(rhd):
    """The kernel timer brackets each kernel with events (plain launches); results are those of the
    graph-replayed run, and the algorithmic bytes follow the arrays the grid carries."""
    case = wl.parity_case("ktime", (40, 24, 36), bc="periodic", exchange="full", beta_tau=True, n_sub=3, seed=35,
                          precision="split")
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(3, case["chat"], case["dt"])
    ref = snapshot(g)
    g.close()
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.set_kernel_timing(True)
    g.radiation_subcycle(3, case["chat"], case["dt"])
    kt = g.kernel_times()
    out = snapshot(g)
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k
    ncell = 40 * 24 * 36
    assert set(kt) == {"twopass_predictor_split", "twopass_corrector_split"}
    # predictor: FP32 state mirror 16 + interleaved FP32 gas 16 in, U^{m+1/2} 16 out; corrector:
    # U^{m+1/2} 16 + U^m 32 + gas 16 + T 8 in, U^{m+1} 32 + T 8 + mirror 16 out (FULL exchange)
    assert kt["twopass_predictor_split"]["alg_bytes_per_launch"] == ncell * (16 + 16 + 16)
    assert kt["twopass_corrector_split"]["alg_bytes_per_launch"] == ncell * (16 + 32 + 16 + 8 + 32 + 8 + 16)
    for v in kt.values():
        assert v["launches"] == 3 and v["total_ms"] > 0
    g.radiation_subcycle(2, case["chat"], case["dt"])
    kt2 = g.kernel_times()  # a new interval
    assert all(v["launches"] == 2 for v in kt2.values())
    g.set_kernel_timing(False)
    g.radiation_subcycle(1, case["chat"], case["dt"])
    assert g.kernel_times() == {}
    g.close()
