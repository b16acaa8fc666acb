"""Chebyshev smoother on the GPU (smoother = 1) against the oracle.

The paper smooths with a block-Jacobi-preconditioned Chebyshev iteration
(Sec. 5.2.1); here it is tuned to an ellipse around the spectrum of D^-1 S
that the library estimates at condensation by Arnoldi.

* The estimate: the GPU's Ritz values (FP64 Arnoldi, classical Gram-Schmidt
  twice, deterministic start vector) equal the oracle's (modified
  Gram-Schmidt, same start vector) and so does the fitted ellipse.
* One preconditioner application with a given ellipse equals the oracle's
  (1e-12 FP64, 1e-5 FP32), sweep counts (2,2), (3,3), (1,1), (0,2), (3,0).
* Solves with the estimated ellipse reach the oracle's direct solution
  (1e-10 at rtol 1e-13) with the oracle's iteration count (within one).
* Under strong rotation (max |f| tau = 8.3 on the r = 4 sphere), damped
  block-Jacobi (omega = 2/3) stops converging, the Chebyshev smoother
  converges (FP64 and mixed) to the oracle's solution.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem
from oracle.solver import TwoLevelPreconditioner, arnoldi_ritz, chebyshev_ellipse, chebyshev_start_vector, gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build
    build.build()


def _case(kind, p, courant=8.0, seed=0):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    tau = courant * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(seed)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    return mesh, prob, (tau, g, H, f), ru, rh


def _solver(mesh, p, tau, g, H, f, **kw):
    from paper_2004_09389_gb300 import HDGSolver
    return HDGSolver(mesh, p, tau, g, H, f_vertex=f, smoother=1, **kw)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _match(a, b):
    return max(np.abs(a[:, None] - b[None, :]).min(axis=1).max(), np.abs(b[:, None] - a[None, :]).min(axis=1).max())


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("sphere", 2)])
def test_estimate_matches_oracle(kind, p):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, cheb_steps=12)
    (theta, delta2), ritz = s.chebyshev()
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S)
    ritz0 = arnoldi_ritz(lambda v: pc.Dinv @ (S @ v), chebyshev_start_vector(prob.n_trace), 12)
    assert len(ritz) == len(ritz0)
    assert _match(ritz, ritz0) <= 1e-8 * np.abs(ritz0).max()
    t0, d0 = chebyshev_ellipse(ritz0)
    assert theta == pytest.approx(t0, rel=1e-8) and delta2 == pytest.approx(d0, rel=1e-6, abs=1e-8)
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("sphere", 2)])
@pytest.mark.parametrize("n_pre,n_post", [(2, 2), (3, 3), (1, 1), (0, 2), (3, 0)])
def test_precond_matches_oracle(kind, p, n_pre, n_post):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    cheb = (1.15, -0.6)
    s = _solver(mesh, p, tau, g, H, f, n_pre=n_pre, n_post=n_post, cheb_theta=cheb[0], cheb_delta2=cheb[1])
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), n_pre=n_pre, n_post=n_post, smoother="chebyshev",
                                cheb=cheb)
    v = np.random.default_rng(2).standard_normal(prob.n_trace)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.precond_apply_dev(torch.from_numpy(v).cuda(), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), pc(v)) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 3), ("sphere", 2)])
def test_precond32_matches_oracle(kind, p):
    from paper_2004_09389_gb300 import HDG_MIXED_FP32
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    cheb = (1.2, 0.3)
    s = _solver(mesh, p, tau, g, H, f, precision=HDG_MIXED_FP32, cheb_theta=cheb[0], cheb_delta2=cheb[1])
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), smoother="chebyshev", cheb=cheb)
    v = np.random.default_rng(3).standard_normal(prob.n_trace)
    z = torch.empty(prob.n_trace, dtype=torch.float32, device="cuda")
    s.precond_apply32_dev(torch.from_numpy(v.astype(np.float32)).cuda(), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), pc(v.astype(np.float32).astype(np.float64))) <= 1e-5
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 3)])
def test_solve_matches_oracle(kind, p):
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-13)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-13
    for a, b in ((lam, lam0.reshape(lam.shape)), (u, u0), (h, h0)):
        assert _rel(a, b) <= 1e-10
    s.close()
    s8 = _solver(mesh, p, tau, g, H, f, rtol=1e-8)
    _, info8 = s8.solve(ru, rh)
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S, smoother="chebyshev", cheb=s8.chebyshev()[0])
    _, info0 = gmres(lambda v: S @ v, prob.condensed_rhs(ru, rh), pc, restart=30, rtol=1e-8)
    assert abs(info8["iters"] - info0["iters"]) <= 1
    s8.close()


def test_strong_rotation_converges_with_chebyshev():
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32
    R, om = 6.371e6, 7.292e-5
    mesh = I.sphere_hierarchy(4, R, r_coarsest=1)
    g, H, p = 9.81, 7500.0, 2
    tau = 32.0 * mesh.h / np.sqrt(g * H)
    f = I.coriolis_sphere(mesh, om)
    assert 8.0 < np.abs(f).max() * tau < 8.5
    ru, rh = I.spherical_harmonic_rhs(mesh, p, 3, lmax=16)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    jac = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-8, max_iter=300)
    _, info_j = jac.solve(ru, rh, allow_fail=True)
    jac.close()
    assert info_j["status"] != 0                          # omega = 2/3 block-Jacobi: no convergence
    for prec, tol in ((0, 1e-8), (HDG_MIXED_FP32, 1e-6)):
        s = _solver(mesh, p, tau, g, H, f, rtol=1e-10, max_iter=300, precision=prec)
        assert s.chebyshev()[0][1] < 0                    # a tall ellipse
        lam, info = s.solve(ru, rh)
        u, h = s.recover()
        assert info["status"] == 0 and info["true_rel_res"] <= 1e-10
        for a, b in ((u, u0), (h, h0)):
            assert _rel(a, b) <= tol
        s.close()
