"""GPU: checkpoint / resume.  A run interrupted by Grid.checkpoint and continued from Grid.restore in a
new context gives bit for bit the state of the uninterrupted run (split and FP64 paths, with a
Dirichlet face and the FULL exchange so that E, F and T all evolve)."""
import numpy as np
import pytest

from paper_1306_0010_gb300 import workloads as wl

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


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_resume_is_bitwise(rhd, tmp_path, precision):
    case = wl.parity_case("ckpt", (24, 20, 18), bc=(["dirichlet", "periodic", "reflect"],
                                                    ["outflow", "periodic", "outflow"]),
                          dirichlet=([[1.5, 0.3, 0.0, 0.0], [0.0] * 4, [0.0] * 4], [[0.0] * 4] * 3),
                          exchange="full", beta_tau=True, with_j=True, n_sub=4, seed=21, precision=precision)
    a = rhd.Grid(case["desc"])
    a.load_case(case)
    a.radiation_subcycle(4, case["chat"], case["dt"])
    ref = a.get_moments()
    ref["T"] = a.get_gas_state()
    a.close()

    b = rhd.Grid(case["desc"])
    b.load_case(case)
    b.radiation_subcycle(2, case["chat"], case["dt"])
    path = str(tmp_path / "state.npz")
    b.checkpoint(path)
    b.close()
    c = rhd.Grid.restore(path)
    c.radiation_subcycle(2, case["chat"], case["dt"])
    out = c.get_moments()
    out["T"] = c.get_gas_state()
    c.close()
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k


def test_conserved_variables_roundtrip(rhd):
    """get_conserved returns (E, F/c) exactly as held; set_conserved gives them back unchanged."""
    case = wl.parity_case("cons", (16, 12, 10), n_sub=1, seed=22, precision="split")
    g = rhd.Grid(case["desc"])
    g.load_case(case)
    g.radiation_subcycle(1, case["chat"], case["dt"])
    cons = g.get_conserved()
    mom = g.get_moments()
    c = case["desc"]["c"]
    assert np.array_equal(cons["E"], mom["E"])
    for d in "xyz":
        assert np.array_equal(cons["G" + d] * c, mom["F" + d])  # get_moments forms F = c G
    h = rhd.Grid(case["desc"])
    h.load_case(case)
    h.set_conserved(cons["E"], cons["Gx"], cons["Gy"], cons["Gz"])
    back = h.get_conserved()
    for k in cons:
        assert np.array_equal(back[k], cons[k]), k
    g.close()
    h.close()
