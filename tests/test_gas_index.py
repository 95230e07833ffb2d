"""Host checks of the gas-step kernels' index arithmetic (no GPU): gas_index_check.cpp enumerates every
index the kernels compute, through the same functions, over whole grids of many shapes and boundary
conditions and checks that each lies inside its array; and the kernels' ghost rule along one axis equals
the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import gas as ogas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BC = ["periodic", "outflow", "reflect", "dirichlet"]


@pytest.fixture(scope="module")
def checker():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    cuda_inc = None
    for cand in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if os.path.exists(os.path.join(cand, "cuda_runtime.h")):
            cuda_inc = cand
            break
    if cuda_inc is None:
        pytest.skip("no CUDA headers")
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "gas_index_check")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(ROOT, "paper_1306_0010_gb300", "csrc"), "-I", cuda_inc,
           os.path.join(ROOT, "tests", "gas_index_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_every_kernel_index_is_in_bounds(checker):
    r = subprocess.run([checker], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert r.stdout.startswith("ok ")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_ghost_rule_equals_the_oracles(checker, n):
    for lo in range(4):
        for hi in range(4):
            r = subprocess.run([checker, "axis", str(n), str(lo), str(hi), "3"], capture_output=True, text=True)
            got = np.array([[float(v) for v in line.split()] for line in r.stdout.split("\n") if line.strip()])
            idx, sgn = ogas.axis_map(n, 3, BC[lo], BC[hi])
            assert np.array_equal(got[:, 1], idx), (n, lo, hi)
            assert np.array_equal(got[:, 2], sgn), (n, lo, hi)
