"""The library's host-side spectral estimate for the Chebyshev smoother
(csrc/spectrum.cpp), on the CPU: eigenvalues of small upper Hessenberg
matrices (real spectra, complex-conjugate pairs, repeated eigenvalues,
Arnoldi matrices of a rotating trace operator) against NumPy, and the ellipse
fit against the same fit written out in the test."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2004_09389_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("spectrum") / "libspectrum.so")
    cmd = [nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-x", "cu", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, os.path.join(ROOT, "tests", "spectrum_check.cpp"), os.path.join(CSRC, "spectrum.cpp"),
           "-o", out, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    L = C.CDLL(out)
    L.hess_eigs.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.ellipse_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p]
    return L


def _eigs(lib, H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    re, im = np.empty(n), np.empty(n)
    lib.hess_eigs(H.ctypes.data, n, re.ctypes.data, im.ctypes.data)
    return re + 1j * im


def _match(a, b):
    """Largest distance from an eigenvalue of b to the nearest one of a, both ways."""
    d1 = np.abs(a[:, None] - b[None, :]).min(axis=1).max()
    d2 = np.abs(b[:, None] - a[None, :]).min(axis=1).max()
    return max(d1, d2)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 20, 40])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_hessenberg(lib, n, seed):
    H = np.triu(np.random.default_rng(seed).standard_normal((n, n)), -1)
    ref = np.linalg.eigvals(H)
    assert _match(_eigs(lib, H), ref) <= 1e-9 * max(1.0, np.abs(ref).max())


def test_structured_spectra(lib):
    # rotation blocks: pure imaginary pairs; a Jordan-like repeated eigenvalue; a symmetric tridiagonal
    R = np.zeros((6, 6))
    for k, w in enumerate((1.0, 2.5, 0.3)):
        R[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[0.5, -w], [w, 0.5]]
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((6, 6)))
    import scipy.linalg as sla
    Hh = sla.hessenberg(Q @ R @ Q.T)
    assert _match(_eigs(lib, Hh), np.linalg.eigvals(R)) <= 1e-9
    T = np.diag(np.full(10, 2.0)) + np.diag(np.full(9, -1.0), 1) + np.diag(np.full(9, -1.0), -1)
    assert _match(_eigs(lib, T), np.linalg.eigvalsh(T).astype(complex)) <= 1e-10
    J = np.diag(np.full(5, 1.5)) + np.diag(np.full(4, 1e-3), -1)
    assert _match(_eigs(lib, J), np.full(5, 1.5 + 0j)) <= 1e-2     # defective: O(eps^(1/5)) sensitivity


def _fit(z, lower=0.1, grow=1.1):
    b = grow * z.real.max()
    a = lower * b
    d, A = 0.5 * (a + b), 0.5 * (b - a)
    q = 1.0 - ((z.real - d) / A) ** 2
    sel = (z.real >= a) & (q > 1e-3)
    B2 = (grow ** 2) * (np.max(z.imag[sel] ** 2 / q[sel]) if sel.any() else 0.0)
    return d, A * A - B2


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_ellipse_fit(lib, seed):
    rng = np.random.default_rng(seed)
    z = rng.uniform(0, 2, 12) + 1j * rng.uniform(-3, 3, 12)
    z = np.concatenate([z, z.conj()])
    out = np.empty(2)
    re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)     # kept alive across the call
    lib.ellipse_fit(re.ctypes.data, im.ctypes.data, len(z), 0.1, 1.1, out.ctypes.data)
    assert out == pytest.approx(_fit(z), rel=1e-13)
