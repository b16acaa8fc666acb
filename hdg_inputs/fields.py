"""Right-hand sides and Coriolis values sampled on the DG input layout.

Input layout (shared contract of the library):

* ``r_u`` is float64 ``[n_cells][2][n_p]`` and ``r_h`` float64
  ``[n_cells][n_p]`` with ``n_p = (p+1)(p+2)/2``: nodal values of the
  right-hand-side functions at the equispaced nodes of each cell.
* Node ``k`` of a cell runs row by row: for ``b = 0..p``, ``a = 0..p-b``, the
  node is ``X0 + (a/p)(X1-X0) + (b/p)(X2-X0)`` with ``X0, X1, X2`` the
  (unwrapped) cell vertices.
* Velocity components are Cartesian on the flat square.  On the sphere they
  are taken in the cell frame ``e1 = (X1-X0)/|X1-X0|``,
  ``e2 = n x e1`` with ``n`` the unit normal of the flat cell.

The generators draw every random number from ``numpy.random.default_rng``
with an explicit seed.
"""
from __future__ import annotations

import math

import numpy as np

from .meshes import Mesh


def _node_pattern(p: int) -> np.ndarray:
    pts = [(a / p, b / p) for b in range(p + 1) for a in range(p + 1 - b)]
    return np.array(pts, dtype=np.float64)


def dg_node_positions(mesh: Mesh, p: int) -> np.ndarray:
    """Coordinates of the DG nodes, float64 ``[n_cells, n_p, dim]``."""
    x = mesh.cell_coords()
    ab = _node_pattern(p)
    return (x[:, None, 0, :] + ab[None, :, 0:1] * (x[:, None, 1, :] - x[:, None, 0, :])
            + ab[None, :, 1:2] * (x[:, None, 2, :] - x[:, None, 0, :]))


def cell_frames(mesh: Mesh) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(e1, e2, n) per cell, each float64 ``[n_cells, 3]`` (sphere meshes)."""
    x = mesh.cell_coords()
    d1 = x[:, 1] - x[:, 0]
    d2 = x[:, 2] - x[:, 0]
    e1 = d1 / np.linalg.norm(d1, axis=1, keepdims=True)
    n = np.cross(d1, d2)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    return e1, e2, n


# --------------------------------------------------------------------------
# manufactured smooth solution on the periodic square
# --------------------------------------------------------------------------

def manufactured_solution(xy: np.ndarray, side: float, c: float, H: float):
    """``h* = sin(kx) cos(ky)``, ``u* = (c/H)(cos kx sin ky, sin kx cos ky)``, k = 2 pi / side."""
    k = 2.0 * math.pi / side
    x, y = xy[..., 0], xy[..., 1]
    h = np.sin(k * x) * np.cos(k * y)
    ux = (c / H) * np.cos(k * x) * np.sin(k * y)
    uy = (c / H) * np.sin(k * x) * np.cos(k * y)
    return ux, uy, h


def manufactured_rhs(mesh: Mesh, p: int, tau: float, g: float, H: float, f: float):
    """RHS functions that make the manufactured pair an exact solution of
    ``u + tau (f u_perp + g grad h) = r_u``, ``h + tau H div u = r_h`` (constant f),
    sampled at the DG nodes.  Returns ``(r_u [N,2,n_p], r_h [N,n_p])``."""
    assert mesh.dim == 2
    c = math.sqrt(g * H)
    side = mesh.side
    k = 2.0 * math.pi / side
    xy = dg_node_positions(mesh, p)
    ux, uy, h = manufactured_solution(xy, side, c, H)
    x, y = xy[..., 0], xy[..., 1]
    dhx = k * np.cos(k * x) * np.cos(k * y)
    dhy = -k * np.sin(k * x) * np.sin(k * y)
    divu = (c / H) * (-2.0 * k) * np.sin(k * x) * np.sin(k * y)
    rux = ux + tau * (f * (-uy) + g * dhx)
    ruy = uy + tau * (f * ux + g * dhy)
    rh = h + tau * H * divu
    return np.stack([rux, ruy], axis=1), rh


def add_noise(r: np.ndarray, std: float, seed: int) -> np.ndarray:
    """Add independent N(0, std^2) noise to every nodal value."""
    rng = np.random.default_rng(seed)
    return r + std * rng.standard_normal(r.shape)


# --------------------------------------------------------------------------
# Gaussian random fields with a k^-3 power spectrum (periodic square)
# --------------------------------------------------------------------------

def _gaussian_grid(rng, grid: int, kmin: float, kmax: float, slope: float) -> np.ndarray:
    kx = np.fft.fftfreq(grid, d=1.0 / grid)
    ky = np.fft.rfftfreq(grid, d=1.0 / grid)
    kk = np.sqrt(kx[:, None] ** 2 + ky[None, :] ** 2)
    amp = np.zeros_like(kk)
    band = (kk >= kmin) & (kk <= kmax)
    amp[band] = kk[band] ** (slope / 2.0)
    spec = amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape))
    fld = np.fft.irfft2(spec, s=(grid, grid))
    fld -= fld.mean()
    fld /= np.sqrt(np.mean(fld ** 2))
    return fld


def _bilinear_periodic(fld: np.ndarray, xy: np.ndarray, side: float) -> np.ndarray:
    grid = fld.shape[0]
    s = (xy / side) * grid
    i0 = np.floor(s).astype(np.int64)
    t = s - i0
    ix0, iy0 = i0[..., 0] % grid, i0[..., 1] % grid
    ix1, iy1 = (ix0 + 1) % grid, (iy0 + 1) % grid
    tx, ty = t[..., 0], t[..., 1]
    # fld is indexed [x, y]
    return ((1 - tx) * (1 - ty) * fld[ix0, iy0] + tx * (1 - ty) * fld[ix1, iy0]
            + (1 - tx) * ty * fld[ix0, iy1] + tx * ty * fld[ix1, iy1])


def gaussian_field_rhs(mesh: Mesh, p: int, seed: int, grid: int = 1024,
                       kmin: float = 1.0, kmax: float = 128.0, slope: float = -3.0):
    """Three independent zero-mean, unit-RMS Gaussian fields with
    ``|g(k)|^2 ~ |k|^slope`` on ``kmin <= |k| <= kmax`` (periodic), synthesised
    on a ``grid^2`` FFT grid and bilinearly interpolated at the DG nodes.
    Returns ``(r_u [N,2,n_p], r_h [N,n_p])``."""
    assert mesh.dim == 2
    rng = np.random.default_rng(seed)
    xy = dg_node_positions(mesh, p)
    out = [_bilinear_periodic(_gaussian_grid(rng, grid, kmin, kmax, slope), xy, mesh.side)
           for _ in range(3)]
    return np.stack(out[:2], axis=1), out[2]


# --------------------------------------------------------------------------
# random spherical-harmonic fields (sphere)
# --------------------------------------------------------------------------

def _sh_coefficients(rng, lmax: int, slope: float) -> np.ndarray:
    """Random coefficients of one field, drawn in the order (m = 0..lmax, then
    l = max(m, 1)..lmax; cos then sin term): array [lmax + 1 (m), lmax + 1 (l), 2],
    zero where unused; standard deviation l^(slope / 2)."""
    c = np.zeros((lmax + 1, lmax + 1, 2))
    for m in range(0, lmax + 1):
        for l in range(max(m, 1), lmax + 1):
            sd = l ** (slope / 2.0)
            c[m, l, 0] = sd * rng.standard_normal()
            if m > 0:
                c[m, l, 1] = sd * rng.standard_normal()
    return c


def _sh_sums(lon: np.ndarray, colat: np.ndarray, coefs: list, chunk: int = 65536) -> list:
    """Sums of real, fully normalised spherical harmonics 1 <= l <= lmax, one
    per coefficient array of ``_sh_coefficients``, at the given directions.
    Associated Legendre values come from the standard three-term recurrences in
    l at fixed m, evaluated once per order for all the fields."""
    lmax = coefs[0].shape[0] - 1
    C = np.stack(coefs)                                  # [F, m, l, 2]
    flat_lon, flat_colat = lon.ravel(), colat.ravel()
    outs = np.zeros((len(coefs), flat_lon.size))
    for a in range(0, flat_lon.size, chunk):
        x = np.cos(flat_colat[a:a + chunk])
        s = np.sin(flat_colat[a:a + chunk])
        ln = flat_lon[a:a + chunk]
        pmm = np.ones_like(x)                            # \bar P_0^0
        for m in range(0, lmax + 1):
            if m == 1:
                pmm = math.sqrt(3.0) * s
            elif m > 1:
                pmm = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
            P = np.empty((lmax + 1 - m, x.size))       # rows l = m .. lmax
            P[0] = pmm
            if m + 1 <= lmax:
                P[1] = math.sqrt(2.0 * m + 3.0) * x * pmm
            for l in range(m + 2, lmax + 1):
                a_ = math.sqrt((2.0 * l - 1.0) * (2.0 * l + 1.0) / ((l - m) * (l + m)))
                b_ = math.sqrt((2.0 * l + 1.0) * (l + m - 1.0) * (l - m - 1.0)
                               / ((l - m) * (l + m) * (2.0 * l - 3.0)))
                P[l - m] = a_ * x * P[l - m - 1] - b_ * P[l - m - 2]
            A = C[:, m, m:, 0] @ P                       # [F, chunk]
            outs[:, a:a + chunk] += A * np.cos(m * ln)
            if m > 0:
                outs[:, a:a + chunk] += (C[:, m, m:, 1] @ P) * np.sin(m * ln)
    return [o.reshape(lon.shape) for o in outs]


def spherical_harmonic_rhs(mesh: Mesh, p: int, seed: int, lmax: int = 64, slope: float = -3.0):
    """``r_h``: a random SH field up to degree lmax with coefficient variance
    ``l^slope``; ``r_u``: three such fields as Cartesian components, projected
    onto each cell's frame.  Evaluated at the radial projection of each DG
    node; each field is scaled to unit RMS over the nodes."""
    assert mesh.dim == 3
    rng = np.random.default_rng(seed)
    xyz = dg_node_positions(mesh, p)
    rr = np.linalg.norm(xyz, axis=-1)
    colat = np.arccos(np.clip(xyz[..., 2] / rr, -1.0, 1.0))
    lon = np.arctan2(xyz[..., 1], xyz[..., 0])

    coefs = [_sh_coefficients(rng, lmax, slope) for _ in range(4)]
    fields = [v / np.sqrt(np.mean(v ** 2)) for v in _sh_sums(lon, colat, coefs)]
    rh = fields[0]
    vec = np.stack(fields[1:], axis=-1)                  # [N, n_p, 3]
    e1, e2, _ = cell_frames(mesh)
    ru = np.stack([np.einsum("kpd,kd->kp", vec, e1), np.einsum("kpd,kd->kp", vec, e2)], axis=1)
    return ru, rh


# --------------------------------------------------------------------------
# Coriolis parameter at the vertices
# --------------------------------------------------------------------------

def coriolis_flat(mesh: Mesh, f0: float) -> np.ndarray:
    return np.full(mesh.n_vertices, f0, dtype=np.float64)


def coriolis_sphere(mesh: Mesh, omega: float = 7.292e-5) -> np.ndarray:
    """``f = 2 Omega sin(latitude) = 2 Omega z / R`` at each vertex."""
    return 2.0 * omega * mesh.vertex_xyz[:, 2] / mesh.radius
