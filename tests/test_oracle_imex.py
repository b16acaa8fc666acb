"""Pins of the IMEX time-stepping oracle (oracle/imex.py): the theta method
and ARS2(2,3,2) around the implicit solve, Coriolis explicit as in the paper.

* the extracted mass matrix is the oracle's load map, and the HDG route of an
  implicit stage (condense, trace solve, recover) equals the direct sparse
  solve of the standard DG stage system;
* one theta = 1 step with f = 0 is one implicit solve of the hot path
  (tau = dt, right-hand side q0);
* the ARS2 tableau printed in the paper is consistent (row sums equal the
  stage times, weights sum to one, b = last implicit row);
* mass is conserved exactly; for f = 0 the energy (H/g)||u||^2 + ||h||^2 does
  not grow under theta >= 1/2 (the upwind operator is dissipative);
* temporal self-convergence orders: 1 for theta = 1 and for theta = 1/2 with
  the explicit Coriolis term, 2 for theta = 1/2 with f = 0 and for ARS2.
"""
import numpy as np
import pytest

import hdg_inputs as I
from hdg_inputs import fields as F
from oracle import imex
from oracle.hdg import HDGProblem

P, G, H = 2, 1.0, 1.0


@pytest.fixture(scope="module")
def mesh():
    return I.periodic_square_hierarchy(8, n_coarsest=2)


@pytest.fixture(scope="module")
def ops(mesh):
    return imex.IMEXOperators(mesh, P, G, H, I.coriolis_flat(mesh, 2.0))


@pytest.fixture(scope="module")
def ops0(mesh):
    return imex.IMEXOperators(mesh, P, G, H, np.zeros(mesh.n_vertices))


def _random_state(ops, seed=0, mean_h=0.7):
    q = np.random.default_rng(seed).standard_normal(ops.M.shape[0]).reshape(ops.N, 3, ops.np)
    q[:, 2, :] += mean_h
    return q.ravel()


def _smooth_state(mesh, ops):
    xy = F.dg_node_positions(mesh, P)
    h = np.sin(2 * np.pi * xy[..., 0]) * np.cos(2 * np.pi * xy[..., 1])
    u = np.stack([np.cos(2 * np.pi * xy[..., 0]) * np.sin(2 * np.pi * xy[..., 1]),
                  0.3 * np.sin(2 * np.pi * xy[..., 1])], axis=1)
    return np.concatenate([u, h[:, None, :]], axis=1).ravel()


def test_mass_matrix_is_the_load_map(mesh, ops):
    q = _random_state(ops)
    u, h = ops.split(q)
    prob = HDGProblem(mesh, P, 1.0, G, H, np.zeros(mesh.n_vertices), lazy=True)
    assert np.abs(ops.mass(q) - prob.load(u, h).ravel()).max() <= 1e-14 * np.abs(ops.mass(q)).max()


@pytest.mark.parametrize("scheme", ["theta", "ars2"])
def test_hdg_route_equals_direct_route(ops, scheme):
    q, dt = _random_state(ops, 1), 0.05
    if scheme == "theta":
        a, b = imex.theta_step(ops, q, dt, 0.5, "direct"), imex.theta_step(ops, q, dt, 0.5, "hdg")
    else:
        a, b = imex.ars2_step(ops, q, dt, "direct"), imex.ars2_step(ops, q, dt, "hdg")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_implicit_euler_is_one_implicit_solve(mesh, ops0):
    q, dt = _random_state(ops0, 2), 0.07
    q1 = imex.theta_step(ops0, q, dt, 1.0)
    u, h = ops0.split(q)
    (u1, h1), _ = HDGProblem(mesh, P, dt, G, H, np.zeros(mesh.n_vertices)).solve_condensed(u, h)
    ref = np.concatenate([u1, h1[:, None, :]], axis=1).ravel()
    assert np.abs(q1 - ref).max() <= 1e-12 * np.abs(ref).max()


def test_ars2_tableau_is_consistent():
    g, d = imex.ARS2_GAMMA, imex.ARS2_DELTA
    a = np.array([[0, 0, 0], [g, 0, 0], [d, 1 - d, 0]])
    at = np.array([[0, 0, 0], [0, g, 0], [0, 1 - g, g]])
    b = np.array([0, 1 - g, g])
    assert np.allclose(a.sum(1), at.sum(1)) and np.allclose(at.sum(1), [0, g, 1])
    assert abs(b.sum() - 1) < 1e-15 and np.allclose(b, at[2])
    assert abs(b @ at.sum(1) - 0.5) < 1e-15 and abs(b @ a.sum(1) - 0.5) < 1e-15    # second-order conditions
    assert abs(g - (1 - 2 ** -0.5)) < 1e-15 and abs(d + 2 * 2 ** 0.5 / 3) < 1e-15


@pytest.mark.parametrize("scheme", ["theta", "ars2"])
def test_mass_is_conserved(ops, scheme):
    q = _random_state(ops, 3)
    m0 = ops.integral_of_h(q)
    for _ in range(8):
        q = imex.theta_step(ops, q, 0.05, 0.5) if scheme == "theta" else imex.ars2_step(ops, q, 0.05)
    assert abs(ops.integral_of_h(q) - m0) <= 1e-12 * abs(m0)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_energy_does_not_grow_without_rotation(ops0, theta):
    q = _random_state(ops0, 4)
    E = [ops0.energy(q)]
    for _ in range(8):
        q = imex.theta_step(ops0, q, 0.05, theta)
        E.append(ops0.energy(q))
    assert all(E[i + 1] <= E[i] * (1 + 1e-13) for i in range(8))
    assert E[-1] < E[0]


@pytest.mark.parametrize("case,order", [("theta1", 1), ("theta_half_rotating", 1), ("theta_half_f0", 2),
                                        ("ars2", 2)])
def test_temporal_order(mesh, ops, ops0, case, order):
    T = 0.4
    q0 = _smooth_state(mesh, ops)

    def run(n):
        q, dt = q0.copy(), T / n
        for _ in range(n):
            if case == "theta1":
                q = imex.theta_step(ops, q, dt, 1.0)
            elif case == "theta_half_rotating":
                q = imex.theta_step(ops, q, dt, 0.5)
            elif case == "theta_half_f0":
                q = imex.theta_step(ops0, q, dt, 0.5)
            else:
                q = imex.ars2_step(ops, q, dt)
        return q

    q16, q32, q64 = run(16), run(32), run(64)
    ratio = np.linalg.norm(q16 - q32) / np.linalg.norm(q32 - q64)
    lo, hi = (1.5, 2.6) if order == 1 else (3.3, 4.8)
    assert lo <= ratio <= hi, ratio


@pytest.mark.parametrize("scheme", ["theta", "ars2"])
def test_sphere_routes_and_mass(scheme):
    """The same two pins on an icosahedral sphere (cells in their own tangent
    frames, f = 2 Omega sin(latitude))."""
    sph = I.sphere_hierarchy(1, 1.0, r_coarsest=0)
    ops_s = imex.IMEXOperators(sph, P, G, H, I.coriolis_sphere(sph, 0.8))
    q, dt = _random_state(ops_s, 5), 0.04
    m0 = ops_s.integral_of_h(q)
    if scheme == "theta":
        a, b = imex.theta_step(ops_s, q, dt, 0.5, "direct"), imex.theta_step(ops_s, q, dt, 0.5, "hdg")
    else:
        a, b = imex.ars2_step(ops_s, q, dt, "direct"), imex.ars2_step(ops_s, q, dt, "hdg")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    assert abs(ops_s.integral_of_h(a) - m0) <= 1e-12 * abs(m0)


def test_general_driver_reproduces_ars2(ops):
    q, dt = _random_state(ops, 6), 0.05
    a = imex.ars2_step(ops, q, dt)
    b = imex.imex_rk_step(ops, q, dt, "ARS2")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("name", ["ARS2", "SSP2", "ARS3"])
def test_tableau_order_conditions(name):
    """Weights sum to one and the second-order conditions hold for both parts
    and their coupling (b.c = b.c~ = b~.c = b~.c~ = 1/2)."""
    a, at, b, bt = (np.asarray(x, float) for x in imex.TABLEAUX[name])
    c, ct = a.sum(1), at.sum(1)
    assert abs(b.sum() - 1) < 1e-14 and abs(bt.sum() - 1) < 1e-14
    for u in (b, bt):
        for v in (c, ct):
            assert abs(u @ v - 0.5) < 1e-14
    assert np.allclose(np.triu(a), 0) and np.allclose(np.triu(at, 1), 0)    # explicit / diagonally implicit


@pytest.mark.parametrize("name,order", [("SSP2", 2), ("ARS3", 3)])
def test_general_driver_orders_and_mass(mesh, ops, name, order):
    T = 0.4
    q0 = _smooth_state(mesh, ops)

    def run(n):
        q = q0.copy()
        for _ in range(n):
            q = imex.imex_rk_step(ops, q, T / n, name)
        return q

    q16, q32, q64 = run(16), run(32), run(64)
    ratio = np.linalg.norm(q16 - q32) / np.linalg.norm(q32 - q64)
    lo, hi = {2: (3.3, 4.8), 3: (6.5, 9.6)}[order]
    assert lo <= ratio <= hi, ratio
    qr = _random_state(ops, 7)
    q1 = imex.imex_rk_step(ops, qr, 0.05, name)
    q1h = imex.imex_rk_step(ops, qr, 0.05, name, route="hdg")
    assert np.abs(q1 - q1h).max() <= 1e-12 * np.abs(q1).max()
    assert abs(ops.integral_of_h(q1) - ops.integral_of_h(qr)) <= 1e-12 * abs(ops.integral_of_h(qr))
