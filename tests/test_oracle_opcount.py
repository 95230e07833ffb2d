"""The op-counting build of the oracle computes exactly what the oracle computes, and its counts
behave as counts of the algorithm's loops (test infrastructure for the ALU roofline)."""
import numpy as np

from oracle import opcount, oracle as orc
from paper_1306_0010_gb300 import workloads as wl


def test_counting_build_is_the_oracle_bitwise():
    case = wl.parity_case("opc", (10, 7, 6), bc=(["outflow", "reflect", "periodic"], ["reflect", "outflow", "periodic"]),
                          exchange="full", beta_tau=True, with_j=True, n_sub=2, seed=3)
    s1, st1, c = opcount.counted_subcycles(case, n_sub=2)
    s2, st2 = orc.subcycles(case, n_sub=2)
    for k in s2:
        assert np.array_equal(s1[k], s2[k]), k
    assert st1 == st2
    assert all(c[k] > 0 for k in ("add", "mul", "div", "sqrt", "cmp"))


def test_counts_scale_with_subcycles_and_are_deterministic():
    case = wl.config4(N=12, n_sub=1)
    _, _, c1 = opcount.counted_subcycles(case, n_sub=1)
    _, _, c1b = opcount.counted_subcycles(case, n_sub=1)
    assert c1 == c1b
    _, _, c2 = opcount.counted_subcycles(case, n_sub=2)
    # the second subcycle repeats the same loops: the sqrt count (outside data-dependent branches)
    # doubles exactly; the rest within the variation of the exchange solve and the limiter
    assert c2["sqrt"] == 2 * c1["sqrt"]
    for k in ("add", "mul", "div"):
        assert abs(c2[k] - 2 * c1[k]) <= 0.02 * c1[k], k


def test_bulk_fit_of_branch_free_classes_is_exact():
    # sqrt is not inside data-dependent branches: its count is an exact cubic in N, so the fitted N^3
    # coefficient is an integer
    r = opcount.bulk_ops_per_cell(lambda N: wl.config4(N=N, n_sub=1), sizes=(8, 10, 12, 14, 16))
    assert abs(r["sqrt"] - round(r["sqrt"])) < 1e-6, r["sqrt"]
    assert 1000 < r["add"] + r["mul"] + r["div"] + r["sqrt"] < 5000
