"""The C-ABI library loads on a machine without a GPU, exports every entry point include/rhd.h
declares, agrees with the binding on struct layouts, and rejects bad arguments before touching
the device.  No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rhd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1306_0010_gb300 import build, rhd

    build.build()
    return rhd.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rhd_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    from paper_1306_0010_gb300 import rhd

    for n in names:
        assert hasattr(lib, n), n
        assert n in rhd._SIGS, f"binding lacks {n}"
    out = subprocess.run(["nm", "-D", "--defined-only", rhd.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r" T (rhd_\w+)", out)))
    assert exported == names


def test_struct_layout_matches_header(tmp_path):
    from paper_1306_0010_gb300 import rhd

    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rhd.h"\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(rhd_grid_desc), offsetof(rhd_grid_desc, cuda_stream),'
                    ' sizeof(rhd_stats), offsetof(rhd_stats, max_f), sizeof(rhd_launch_config),'
                    ' offsetof(rhd_launch_config, ms_per_subcycle)); printf("%zu %zu\\n", sizeof(rhd_kernel_time),'
                    ' offsetof(rhd_kernel_time, alg_bytes_per_launch)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    a, b, c, d, e, f, g, h = (int(v) for v in subprocess.check_output([str(exe)]).split())
    assert g == ctypes.sizeof(rhd.KernelTime) and h == rhd.KernelTime.alg_bytes_per_launch.offset
    assert a == ctypes.sizeof(rhd.GridDesc) and b == rhd.GridDesc.cuda_stream.offset
    assert c == ctypes.sizeof(rhd.Stats) and d == rhd.Stats.max_f.offset
    assert e == ctypes.sizeof(rhd.LaunchConfig) and f == rhd.LaunchConfig.ms_per_subcycle.offset


def test_identification_and_argument_errors(lib):
    from paper_1306_0010_gb300 import rhd, workloads as wl

    assert lib.rhd_abi_version() == 2
    assert lib.rhd_built_arch() == 103
    # NULL out pointer
    desc = rhd.desc_struct(wl.base_desc((8, 8, 8), (0.1, 0.1, 0.1)))
    assert lib.rhd_init_grid(None, ctypes.byref(desc)) == rhd.ERR_ARG
    # invalid descriptors are rejected before any device call
    bad = [
        dict(n=(8, 1, 8)),                     # inactive direction not trailing
        dict(n=(2, 8, 8)),                     # active direction with n < 3
        dict(theta_F=0.0),
        dict(E_floor=0.0),
        dict(gamma=1.0),
        dict(kappa_rho_pow=3),
        dict(cfl=1.5),
    ]
    for kw in bad:
        d = wl.base_desc((8, 8, 8), (0.1, 0.1, 0.1))
        d.update(kw)
        ctx = ctypes.c_void_p()
        st = lib.rhd_init_grid(ctypes.byref(ctx), ctypes.byref(rhd.desc_struct(d)))
        assert st == rhd.ERR_ARG, kw
        assert lib.rhd_last_error(None)
        assert not ctx
    # NULL contexts
    assert lib.rhd_radiation_subcycle(None, 1, 1.0, 0.1) == rhd.ERR_ARG
    assert lib.rhd_destroy(None) == rhd.OK
    assert lib.rhd_gas_step(None, 1.0) == rhd.ERR_ARG
    assert lib.rhd_gas_correct(None) == rhd.ERR_ARG
    assert lib.rhd_get_gas(None, None, None, None, None, None, 0) == rhd.ERR_ARG
    cfg = rhd.LaunchConfig()
    assert lib.rhd_autotune(None, 1.0, 0.1, 1, None, 0, None, None) == rhd.ERR_ARG
    assert lib.rhd_ensemble_autotune(None, 1.0, None, 1, None, 0, None, None) == rhd.ERR_ARG
    assert lib.rhd_get_launch_config(None, ctypes.byref(cfg)) == rhd.ERR_ARG
    assert lib.rhd_set_launch_config(None, ctypes.byref(cfg)) == rhd.ERR_ARG
    assert lib.rhd_set_kernel_timing(None, 1) == rhd.ERR_ARG
    assert lib.rhd_get_kernel_times(None, None, 0, None) == rhd.ERR_ARG
