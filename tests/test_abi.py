"""The C-ABI library loads and exports every function include/igr.h declares
(no compute: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "igr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(igr_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_stage_calls():
    names = declared_functions()
    for fn in ("igr_create", "igr_set_state", "igr_step", "igr_solve_sigma", "igr_rhs",
               "igr_get_state", "igr_destroy"):
        assert fn in names


@pytest.fixture(scope="module")
def libigr():
    from paper_2505_07392_gb300 import build, igr
    if not os.path.exists(igr.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc is not available to build libigr.so")
        build.build()
    return ctypes.CDLL(igr.LIB_PATH)


def test_library_exports_every_declared_function(libigr):
    for name in declared_functions():
        assert hasattr(libigr, name), name


def test_host_only_calls(libigr):
    """Calls that need no GPU: version, invalid-config rejection, memory sizing."""
    from paper_2505_07392_gb300 import igr, inputs
    L = igr.lib()
    assert L.igr_version().decode().startswith("igr-gb300")
    case = inputs.density_wave(32)
    cfg, _ = igr.make_config(case, "f32")
    # 3 states x 5 fields + 2 Sigma + b = 18 words per cell, plus small tables
    n = case.ncells
    assert L.igr_memory_bytes(ctypes.byref(cfg)) >= 18 * 4 * n
    bad, _ = igr.make_config(inputs.density_wave(3), "f32")
    assert L.igr_memory_bytes(ctypes.byref(bad)) == 0
    h = ctypes.c_void_p()
    assert L.igr_create(ctypes.byref(bad), None, None, ctypes.byref(h)) == igr.ERR_INVALID_ARG
    assert b">= 4" in L.igr_last_error(None)
    # inflow is only allowed on -z
    c2 = inputs.blast(16)
    c2.bc = (inputs.INFLOW,) + (inputs.OUTFLOW,) * 5
    cfg2, _ = igr.make_config(c2, "f32")
    assert L.igr_create(ctypes.byref(cfg2), None, None, ctypes.byref(h)) == igr.ERR_INVALID_ARG
    assert b"-z face" in L.igr_last_error(None)
    # host_rk_base: one 5-field state buffer fewer on the device (13 words per cell)
    cfgh, _ = igr.make_config(case, "f16", host_rk_base=True)
    cfgd, _ = igr.make_config(case, "f16")
    state = -(-5 * 2 * n // 256) * 256
    assert L.igr_memory_bytes(ctypes.byref(cfgd)) - L.igr_memory_bytes(ctypes.byref(cfgh)) == state
    cfgh.host_rk_base = 2
    assert L.igr_create(ctypes.byref(cfgh), None, None, ctypes.byref(h)) == igr.ERR_INVALID_ARG
    assert b"host_rk_base" in L.igr_last_error(None)
    # red-black sweeps work in place: one Sigma buffer fewer
    from dataclasses import replace
    cfgr, _ = igr.make_config(replace(case, sigma_solver=1), "f16")
    sig = -(-2 * n // 256) * 256
    assert L.igr_memory_bytes(ctypes.byref(cfgd)) - L.igr_memory_bytes(ctypes.byref(cfgr)) == sig
    # ... and need even periodic axes; only orders 3 and 5 exist
    for bad_case, word in ((replace(inputs.density_wave(31), sigma_solver=1), b"even"),
                           (replace(case, order=4), b"order")):
        cb, _ = igr.make_config(bad_case, "f32")
        assert L.igr_create(ctypes.byref(cb), None, None, ctypes.byref(h)) == igr.ERR_INVALID_ARG
        assert word in L.igr_last_error(None)
    # calls on a NULL context are rejected before any device work
    i = ctypes.c_int()
    assert L.igr_set_conserved(None, None, igr.DT_F32, 1) == igr.ERR_INVALID_ARG
    assert L.igr_step_host(None, None, None, 1, igr.DT_F32) == igr.ERR_INVALID_ARG
    assert L.igr_set_kernel_forms(None, 0, 0) == igr.ERR_INVALID_ARG
    assert L.igr_get_kernel_forms(None, ctypes.byref(i), ctypes.byref(i)) == igr.ERR_INVALID_ARG
    assert L.igr_autotune_batch(None, 3) == igr.ERR_INVALID_ARG
    assert L.igr_step_batch(None, 1) == igr.ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path):
    """With no CUDA library at the configured path the binding raises at its
    first call: there is no CPU fallback."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2505_07392_gb300 import igr, inputs\n"
            "try:\n"
            "    igr.memory_bytes(inputs.density_wave(8))\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % root
    env = dict(os.environ, IGR_LIBRARY=str(tmp_path / "absent" / "libigr.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "is missing" in r.stdout
