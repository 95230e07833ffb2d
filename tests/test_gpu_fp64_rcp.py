"""GPU: the FP64 path's reciprocal and inverse square root (two Newton-Raphson steps on the hardware
approximations) are within two units in the last place of CUDA's correctly rounded 1.0 / x and within
three of 1.0 / sqrt(x) (itself two roundings); x rsqrt(x) on [1, 4], the closure's square root, within
two of sqrt(x)."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1306_0010_gb300", "csrc")


def test_fp64_reciprocal_within_two_ulp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build

    os.makedirs(build.BUILD, exist_ok=True)
    exe = os.path.join(build.BUILD, "fp64_rcp_check")
    subprocess.run([build.nvcc(), "-std=c++17", "-O3", *build.ARCH, "-I", CSRC, os.path.join(HERE, "fp64_rcp_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    fields = dict(zip(out.split()[0::2], (int(v) for v in out.split()[1::2])))
    assert fields["max_ulp"] <= 2, out
    assert fields["max_ulp_rsqrt"] <= 3, out
    assert fields["max_ulp_sqrt14"] <= 2, out
