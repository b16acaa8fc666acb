"""Host logic of the single-CTA coarse cycle, on the CPU: its shared-memory
layout (csrc/layout.cpp) for every admissible first tail level of flat and
sphere hierarchies, FP64 and FP32 values.  tests/tail_layout_check.cpp checks
16-byte alignment, that the pieces follow the level table without overlap and
match its offsets and sizes, that the scratch vectors lie after the staged
image, the rule for staging the coarsest inverse, and the shared-memory limit.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

import hdg_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2004_09389_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tailcheck") / "libtailcheck.so")
    cmd = [nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-x", "cu",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, os.path.join(ROOT, "tests", "tail_layout_check.cpp"),
           os.path.join(CSRC, "layout.cpp"), os.path.join(CSRC, "mesh.cpp"), os.path.join(CSRC, "refelem.cpp"),
           "-o", out, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    lib = C.CDLL(out)
    lib.check_tail_layouts.argtypes = [C.c_void_p, C.c_char_p, C.c_int]
    return lib


@pytest.mark.parametrize("kind,n", [("flat", 24), ("flat", 256), ("sphere", 3), ("sphere", 6)])
def test_tail_layout(checker, kind, n):
    from paper_2004_09389_gb300 import _lib as L
    mesh = (I.periodic_square_hierarchy(n, n_coarsest=3 if n < 64 else 4) if kind == "flat"
            else I.sphere_hierarchy(n, 1.0, r_coarsest=0))
    keep = []
    desc = L.make_mesh_desc(mesh, keep)
    buf = C.create_string_buffer(1 << 16)
    rc = checker.check_tail_layouts(C.addressof(desc), buf, len(buf))
    rep = buf.value.decode()
    assert rc == 0, rep
    assert "first tail level" in rep
