"""GPU: the bounds-checked debug library (librhd_debug.so) on tiny grids (4x3x3, 5x3x3, one-cell-wide
dimensions), ragged tiles, every boundary rule, both precisions, the fused and two-pass kernels,
TMA staging and an ensemble: no kernel index leaves its array, and the results still match the
oracle.  The debug build stands in for a memory checker: its index checks count an out-of-range
index and redirect the access, so a mistake is reported, never a fault."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FP64_TOL = 1e-12


def test_debug_build_finds_no_out_of_range_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1306_0010_gb300 import build

    build.build()
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_sweep.py")], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert lines[0] == {"bounds_checked": 1}
    results = lines[1:]
    assert len(results) >= 14
    for res in results:
        assert res["status"] == 0 and res["bounds_violations"] == 0, res
        tol = FP64_TOL if res["precision"] == "fp64" else res["bound"]  # split: split_bounds.split_bound
        assert res["error"] <= tol, res
