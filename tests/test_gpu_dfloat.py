"""GPU: the double-float operations of the split path's stiff sources (csrc/dfloat.cuh) stay within
small multiples of u^2 = 2^-48 of the FP64 result over 2^20 random operands (a quarter of the sums
nearly cancelling), and the integer FP64 -> FP32 round-to-nearest equals CUDA's conversion bit for bit."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1306_0010_gb300", "csrc")

# relative error bounds in units of u^2 (Joldes, Muller & Popescu 2017 for the compound operations;
# the FP64 reference itself adds about 1/32)
BOUNDS = {"d2df": 1.05, "add_fp": 2.05, "add": 3.05, "add_same": 3.05, "mul_fp": 2.05, "mul": 5.05, "sqr": 5.05,
          "rcp": 4.05}


def test_double_float_operations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build

    os.makedirs(build.BUILD, exist_ok=True)
    exe = os.path.join(build.BUILD, "dfloat_check")
    subprocess.run([build.nvcc(), "-std=c++17", "-O3", *build.ARCH, "-I", CSRC, os.path.join(HERE, "dfloat_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    vals = dict(zip(out.split()[0::2], (float(v) for v in out.split()[1::2])))
    print(out)
    assert vals["rn_miss"] == 0, out
    for k, b in BOUNDS.items():
        assert vals[k] <= b, (k, vals[k], out)
