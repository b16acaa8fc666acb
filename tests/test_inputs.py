"""Pins of the seeded input generators (hdg_inputs/), which both the oracle
and the GPU path consume: mesh counts, orientation, closure and Euler
characteristic; the nested hierarchies' parent maps against vertex positions;
DG node positions; the Coriolis fields; the random fields' statistics and
spectrum; the spherical-harmonic recurrence against SciPy's associated
Legendre functions."""
import math

import numpy as np
import pytest

import hdg_inputs as I
from hdg_inputs import fields as F


def _edges(cells):
    e = np.concatenate([cells[:, [0, 1]], cells[:, [1, 2]], cells[:, [2, 0]]])
    return e


def _check_closed_oriented(cells, n_vertices, euler):
    e = _edges(cells)
    directed = {tuple(x) for x in e}
    assert len(directed) == len(e), "a directed edge appears twice (inconsistent orientation)"
    for a, b in e:
        assert (b, a) in directed, "an edge has only one cell"
    n_edges = len(e) // 2
    assert n_vertices - n_edges + len(cells) == euler


@pytest.mark.parametrize("n", [3, 8, 17])
def test_periodic_square(n):
    m = I.periodic_square(n, side=2.0)
    assert m.n_vertices == n * n and m.n_cells == 2 * n * n
    X = m.vertex_xyz[m.cell_vertices] + m.cell_shift          # unwrapped corners
    area = 0.5 * ((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1])
                  - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1]))
    assert np.allclose(area, 0.5 * (2.0 / n) ** 2)             # all counter-clockwise, equal
    _check_closed_oriented(m.cell_vertices, m.n_vertices, 0)   # a torus


def _periodic_midpoint(a, b, side):
    d = (b - a + side / 2) % side - side / 2                   # shortest periodic difference
    return (a + d / 2) % side


@pytest.mark.parametrize("n,nc", [(16, 2), (24, 3)])
def test_square_hierarchy_parents(n, nc):
    m = I.periodic_square_hierarchy(n, side=1.0, n_coarsest=nc)
    fine = m
    for lev in m.levels:
        par = lev.parent
        assert par.shape == (fine.n_vertices, 2)
        Xf, Xc = fine.vertex_xyz, lev.vertex_xyz
        same = par[:, 0] == par[:, 1]
        assert np.allclose(Xf[same], Xc[par[same, 0]])
        mid = _periodic_midpoint(Xc[par[~same, 0]], Xc[par[~same, 1]], 1.0)
        diff = (Xf[~same] - mid + 0.5) % 1.0 - 0.5
        assert np.abs(diff).max() < 1e-12
        assert same.sum() == lev.n_vertices                    # every coarse vertex is also fine
        fine = lev


@pytest.mark.parametrize("r", [0, 1, 3])
def test_icosahedral_sphere(r):
    R = 6.371e6
    m = I.icosahedral_sphere(r, radius=R)
    assert m.n_vertices == 10 * 4 ** r + 2 and m.n_cells == 20 * 4 ** r
    assert np.allclose(np.linalg.norm(m.vertex_xyz, axis=1), R)
    X = m.vertex_xyz[m.cell_vertices]
    nrm = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    assert (np.einsum("kd,kd->k", nrm, X.sum(1)) > 0).all()   # counter-clockwise seen from outside
    _check_closed_oriented(m.cell_vertices, m.n_vertices, 2)


def test_sphere_hierarchy_parents():
    m = I.sphere_hierarchy(3, 2.0, r_coarsest=0)
    fine = m
    for lev in m.levels:
        par = lev.parent
        Xf, Xc = fine.vertex_xyz, lev.vertex_xyz
        same = par[:, 0] == par[:, 1]
        assert np.allclose(Xf[same], Xc[par[same, 0]])
        mid = Xc[par[~same, 0]] + Xc[par[~same, 1]]
        mid = 2.0 * mid / np.linalg.norm(mid, axis=1, keepdims=True)
        assert np.abs(Xf[~same] - mid).max() < 1e-12
        fine = lev


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dg_nodes_include_the_vertices(p):
    m = I.periodic_square(4, side=1.0)
    xy = F.dg_node_positions(m, p)
    assert xy.shape[:2] == (m.n_cells, (p + 1) * (p + 2) // 2)
    X = m.vertex_xyz[m.cell_vertices] + m.cell_shift
    for v in range(3):                                       # each corner is one of the nodes
        d = np.linalg.norm(xy - X[:, v][:, None, :], axis=-1).min(axis=1)
        assert d.max() < 1e-12


def test_coriolis_fields():
    m = I.icosahedral_sphere(2, radius=3.0)
    om = 7.292e-5
    assert np.allclose(I.coriolis_sphere(m, om), 2 * om * m.vertex_xyz[:, 2] / 3.0)
    q = I.periodic_square(5)
    assert np.allclose(I.coriolis_flat(q, 1e-4), 1e-4)


def test_gaussian_field_statistics_and_spectrum():
    rng = np.random.default_rng(3)
    fld = F._gaussian_grid(rng, 256, 1.0, 64.0, -3.0)
    assert abs(fld.mean()) < 1e-12 and abs(np.sqrt(np.mean(fld ** 2)) - 1.0) < 1e-12
    P = np.abs(np.fft.fft2(fld)) ** 2
    k = np.sqrt(np.fft.fftfreq(256, 1 / 256)[:, None] ** 2 + np.fft.fftfreq(256, 1 / 256)[None, :] ** 2)
    assert P[(k > 64.5)].max() < 1e-18 * P.max()             # nothing outside the band
    kb = np.arange(4, 60)
    pw = np.array([P[(k >= a) & (k < a + 1)].mean() for a in kb])
    slope = np.polyfit(np.log(kb + 0.5), np.log(pw), 1)[0]
    assert abs(slope - (-3.0)) < 0.25                        # mean power per mode in a shell ~ k^slope
    ru, rh = I.gaussian_field_rhs(I.periodic_square(16), 2, seed=1, grid=256, kmax=32.0)
    assert ru.shape == (512, 2, 6) and rh.shape == (512, 6) and np.isfinite(ru).all()


def _normalised_legendre(l, m, x):
    from scipy.special import lpmv
    lognorm = 0.5 * (math.log((2.0 - (m == 0)) * (2 * l + 1)) + math.lgamma(l - m + 1) - math.lgamma(l + m + 1))
    return (-1.0) ** m * lpmv(m, l, x) * math.exp(lognorm)    # Condon-Shortley phase removed


@pytest.mark.parametrize("l,m", [(1, 0), (1, 1), (2, 1), (5, 3), (17, 0), (17, 17), (40, 12), (64, 31), (64, 64)])
def test_spherical_harmonic_recurrence(l, m):
    """_sh_sums with one nonzero coefficient (cos or sin term of degree l,
    order m) equals the fully normalised P_l^m(cos colat) cos / sin (m lon)."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(l * 100 + m)
    colat = np.arccos(rng.uniform(-1, 1, 200))
    lon = rng.uniform(-np.pi, np.pi, 200)
    lmax = 64
    c = np.zeros((lmax + 1, lmax + 1, 2))
    c[m, l, 0] = 1.0
    s = np.zeros_like(c)
    if m > 0:
        s[m, l, 1] = 1.0
    got_c, got_s = F._sh_sums(lon, colat, [c, s])
    ref = _normalised_legendre(l, m, np.cos(colat))
    scale = np.abs(ref).max()
    assert np.abs(got_c - ref * np.cos(m * lon)).max() <= 1e-10 * scale
    if m > 0:
        assert np.abs(got_s - ref * np.sin(m * lon)).max() <= 1e-10 * scale
