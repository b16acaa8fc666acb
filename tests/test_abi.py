"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hdg.h (no GPU needed: nothing is computed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    return sorted(set(re.findall(r"HDG_API\s+[\w\s\*]*?\b(hdg_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2004_09389_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for name in ("hdg_setup", "hdg_condense", "hdg_solve", "hdg_recover", "hdg_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(hdg_\w+)", out))
    assert set(declared_symbols()) <= exported
    # nothing else leaks out of the library
    assert exported == set(declared_symbols())


def test_library_loads_and_binding_matches(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name)
    from paper_2004_09389_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_symbols()
    prm = _lib.default_params()          # host-only call
    assert prm.p == 1 and prm.restart == 30 and abs(prm.omega - 2 / 3) < 1e-15


def test_setup_rejects_bad_arguments_without_gpu(lib_path):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    prm = _lib.default_params()
    prm.p = 7
    h = ctypes.c_void_p()
    rc = lib.hdg_setup(None, ctypes.byref(prm), None, ctypes.byref(h))
    assert rc == _lib.HDG_EINVAL and not h.value
    assert b"p must be" in lib.hdg_last_error(None)
    # the last field of hdg_params reaches the library at the offset the binding uses
    prm = _lib.default_params()
    assert prm.reorth == 0
    prm.reorth = 3
    rc = lib.hdg_setup(None, ctypes.byref(prm), None, ctypes.byref(h))
    assert rc == _lib.HDG_EINVAL and not h.value
    assert b"reorth must be" in lib.hdg_last_error(None)
    # keep_rhs, the struct's last field: 1 by default, 0 or 1 only
    prm = _lib.default_params()
    assert prm.keep_rhs == 1
    prm.keep_rhs = 2
    rc = lib.hdg_setup(None, ctypes.byref(prm), None, ctypes.byref(h))
    assert rc == _lib.HDG_EINVAL and not h.value
    assert b"keep_rhs must be" in lib.hdg_last_error(None)


def test_step_entry_points_reject_a_null_handle_without_gpu(lib_path):
    """Steps 1-3 (one call or separate) check the handle on the host before any
    CUDA call: a NULL handle is HDG_EINVAL."""
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    info = _lib.hdg_solve_info()
    buf = (ctypes.c_double * 8)()
    p = ctypes.addressof(buf)
    assert lib.hdg_solve_recover(None, p, p, p, p, p, ctypes.byref(info)) == _lib.HDG_EINVAL
    assert lib.hdg_solve(None, p, p, p, ctypes.byref(info)) == _lib.HDG_EINVAL
    assert lib.hdg_recover(None, None, None, None, p, p) == _lib.HDG_EINVAL
    assert lib.hdg_recover_dev(None, None, None, None, p, p) == _lib.HDG_EINVAL
