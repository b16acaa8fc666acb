"""Host logic of the patch-fused P1 kernels, on the CPU.

The library's own mesh code (csrc/mesh.cpp, csrc/refelem.cpp) is compiled
with tests/patch_check.cpp, which rebuilds the P1 hierarchy and checks every
index the fused kernels follow: local columns against the level operator,
children slots and weights against the restriction, the per-row copies of
columns and prolongation parents, that every coarse vertex lies in exactly
one patch, every fine vertex in some F0 set and in exactly one owned set, and
the recorded maximum sizes.
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
    out = str(tmp_path_factory.mktemp("patchcheck") / "libpatchcheck.so")
    cmd = [nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-x", "cu",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, os.path.join(ROOT, "tests", "patch_check.cpp"),
           os.path.join(CSRC, "mesh.cpp"), os.path.join(CSRC, "refelem.cpp"), "-o", out, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    lib = C.CDLL(out)
    lib.check_patches.argtypes = [C.c_void_p, C.c_char_p, C.c_int]
    return lib


def _check(lib, mesh):
    from paper_2004_09389_gb300 import _lib as L
    keep = []
    desc = L.make_mesh_desc(mesh, keep)
    buf = C.create_string_buffer(1 << 16)
    rc = lib.check_patches(C.addressof(desc), buf, len(buf))
    return rc, buf.value.decode()


@pytest.mark.parametrize("kind,n", [("flat", 24), ("flat", 256), ("sphere", 3), ("sphere", 6)])
def test_patches_follow_the_level_operators(checker, kind, n):
    mesh = (I.periodic_square_hierarchy(n, n_coarsest=3 if n < 64 else 4) if kind == "flat"
            else I.sphere_hierarchy(n, 6.371e6 if n > 4 else 1.0, r_coarsest=0))
    rc, rep = _check(checker, mesh)
    assert rc == 0, rep
    assert "patches" in rep
