"""Pins of the oracle's learned facet-patch smoother (no GPU).

* the hand-written backward pass equals central finite differences of the loss;
* with zero weights the correction is exactly the damped block-Jacobi step;
* the correction is positively homogeneous of degree one in the residual.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem
from oracle import learned as LN
from oracle.solver import TwoLevelPreconditioner


def _setup(p=1, n=6):
    mesh = I.periodic_square_hierarchy(n, n_coarsest=3)
    prob = HDGProblem(mesh, p, tau=0.2, g=1.0, H=1.0, f_vertex=I.coriolis_flat(mesh, 1.0))
    S = prob.trace_operator().tocsr()
    pc = TwoLevelPreconditioner(prob, mesh, S)
    pp = p + 1
    NF = prob.n_facets
    nbr = np.zeros((NF, 4), int)
    cnt = np.zeros(NF, int)
    # neighbour order of the library: for facet e with cells (K_s, i_s), s = 0, 1,
    # the facets of local edges (i_s + 1 + k) % 3, k = 0, 1
    seen = {}
    for K in range(prob.N):
        for i in range(3):
            e = prob.facet_of[K, i]
            s = seen.get(e, 0)
            seen[e] = s + 1
            for k in range(2):
                nbr[e, 2 * s + k] = prob.facet_of[K, (i + 1 + k) % 3]
    Dinv = np.stack([pc.Dinv[e * pp:(e + 1) * pp][:, e * pp:(e + 1) * pp].toarray() for e in range(NF)])
    return prob, S, pc, nbr, Dinv, pp


def test_backward_matches_finite_differences():
    prob, S, pc, nbr, Dinv, pp = _setup()
    hid = 5
    rng = np.random.default_rng(0)
    theta = 0.3 * rng.standard_normal(LN.n_params(5 * pp, hid, pp))
    R = rng.standard_normal((2, prob.n_trace))
    L0, g = LN.loss_and_grad(theta, R, S, nbr, Dinv, hid, pp, 2.0 / 3.0)
    eps = 1e-6
    for k in rng.choice(theta.size, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (LN.loss_and_grad(tp, R, S, nbr, Dinv, hid, pp, 2 / 3)[0]
              - LN.loss_and_grad(tm, R, S, nbr, Dinv, hid, pp, 2 / 3)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8


def test_zero_weights_give_damped_block_jacobi():
    prob, S, pc, nbr, Dinv, pp = _setup()
    hid = 4
    theta = np.zeros(LN.n_params(5 * pp, hid, pp))
    r = np.random.default_rng(1).standard_normal(prob.n_trace)
    c = LN.correction(theta, r, nbr, Dinv, hid, pp, 2.0 / 3.0)
    assert np.allclose(c, (2.0 / 3.0) * (pc.Dinv @ r), rtol=1e-12, atol=1e-14)


def test_positive_homogeneity():
    prob, S, pc, nbr, Dinv, pp = _setup(p=2)
    hid = 6
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(LN.n_params(5 * pp, hid, pp))
    r = rng.standard_normal(prob.n_trace)
    c1 = LN.correction(theta, r, nbr, Dinv, hid, pp, 2 / 3)
    c2 = LN.correction(theta, 7.5 * r, nbr, Dinv, hid, pp, 2 / 3)
    assert np.allclose(c2, 7.5 * c1, rtol=1e-11, atol=1e-13)
