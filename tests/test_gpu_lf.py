"""Lax-Friedrichs solver on the GPU (flux = 1: vector trace, RT0 coarse space)
against the Lax-Friedrichs oracle (oracle/lf.py): Eq. bilinear_HDG_lax with the
ABCM operators of App. B, the RT0 coarse space and Eq. coarse_problem_LF of
Sec. 4.4, on flat periodic meshes of several 256-thread tiles with a ragged
tail, p = 1 and 2.

* per-cell S_K (6(p+1) x 6(p+1)), the trace operator and the condensed RHS
  equal the oracle's to 1e-12;
* the coarse solve's ellipse (Arnoldi Ritz values of D_c^-1 S_c) equals the
  oracle's; one preconditioner application with the same ellipse equals the
  oracle's to 1e-12 (block-Jacobi and Chebyshev smoothers, with and without
  rotation in the coarse operator);
* the solve (rtol 1e-13) and the recovery equal the oracle's direct solution
  to 1e-10 per field; iteration counts to 1e-8 agree within one;
* configurations outside the variant's scope are rejected on the host.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.lf import LFProblem, LFTwoLevelPreconditioner
from oracle.solver import arnoldi_ritz, chebyshev_ellipse, chebyshev_start_vector, gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build
    build.build()


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _case(p, n=12, f0=1.0, courant=4.0):
    mesh = I.periodic_square_hierarchy(n, n_coarsest=3)     # 288 cells, 432 facets at n = 12
    g, H = 1.3, 0.7
    tau = courant * mesh.h / np.sqrt(g * H)
    f = I.coriolis_flat(mesh, f0)
    prob = LFProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(p)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    return mesh, prob, (tau, g, H, f), ru, rh


def _solver(mesh, p, tau, g, H, f, **kw):
    from paper_2004_09389_gb300 import HDGSolver
    return HDGSolver(mesh, p, tau, g, H, f_vertex=f, flux=1, **kw)


@pytest.mark.parametrize("p", [1, 2])
def test_operators_match_oracle(p):
    mesh, prob, (tau, g, H, f), ru, rh = _case(p)
    s = _solver(mesh, p, tau, g, H, f)
    S = s.cell_schur()
    S0 = np.stack([prob.cell_schur(K) for K in range(prob.N)])
    assert S.shape == S0.shape and np.abs(S - S0).max() <= 1e-12 * np.abs(S0).max()
    x = np.random.default_rng(3).standard_normal(prob.n_trace)
    y = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.trace_apply_dev(torch.from_numpy(x).cuda(), y)
    gd = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.condensed_rhs_dev(torch.from_numpy(ru).cuda(), torch.from_numpy(rh).cuda(), gd)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy(), prob.trace_operator() @ x) <= 1e-12
    assert _rel(gd.cpu().numpy(), prob.condensed_rhs(ru, rh)) <= 1e-12
    s.close()


@pytest.mark.parametrize("p,smoother,coarse_mode", [(1, 0, 0), (2, 0, 0), (2, 1, 0), (1, 0, 1)])
def test_precond_matches_oracle(p, smoother, coarse_mode):
    mesh, prob, (tau, g, H, f), _, _ = _case(p)
    kw = dict(smoother=smoother, coarse_mode=coarse_mode, n_coarse=12)
    if smoother:
        kw.update(cheb_theta=1.1, cheb_delta2=0.5)
    s = _solver(mesh, p, tau, g, H, f, **kw)
    S = prob.trace_operator()
    if coarse_mode == 1:
        # the coarse operator without rotation: the oracle's with f = 0 in it
        prob_nf = LFProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=np.zeros(mesh.n_vertices))
        from oracle.lf import rt0_operator
        Sc_nf = rt0_operator(prob_nf)
    ell_c, ritz_c = s.chebyshev(coarse=True)
    pc = LFTwoLevelPreconditioner(prob, S, coarse="chebyshev", n_coarse=12, cheb_c=ell_c)
    if coarse_mode == 1:
        pc.Sc, pc.dc = Sc_nf.tocsr(), 1.0 / Sc_nf.diagonal()
    # the device's coarse estimate is the oracle's (same start vector, same fit)
    ritz0 = arnoldi_ritz(lambda v: pc.dc * (pc.Sc @ v), chebyshev_start_vector(prob.n_facets), 20)
    assert len(ritz_c) == len(ritz0)
    assert max(np.abs(ritz_c[:, None] - ritz0[None, :]).min(axis=1)) <= 1e-8 * np.abs(ritz0).max()
    t0, d0 = chebyshev_ellipse(ritz0)
    assert ell_c[0] == pytest.approx(t0, rel=1e-8) and ell_c[1] == pytest.approx(d0, rel=1e-6, abs=1e-8)
    if smoother:
        # the oracle's Chebyshev smoother on the 2(p+1) blocks, same ellipse
        from oracle.solver import TwoLevelPreconditioner
        th, d2 = 1.1, 0.5

        def smooth(b, x, n, _pc=pc):
            if n == 0:
                return x
            s_prev = 1.0 / th
            d = s_prev * (_pc.Dinv @ (b - S @ x))
            x = x + d
            for _ in range(1, n):
                si = 1.0 / (2.0 * th - d2 * s_prev)
                d = d2 * si * s_prev * d + 2.0 * si * (_pc.Dinv @ (b - S @ x))
                x = x + d
                s_prev = si
            return x
        pc.smooth = smooth
    v = np.random.default_rng(4).standard_normal(prob.n_trace)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.precond_apply_dev(torch.from_numpy(v).cuda(), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), pc(v)) <= 1e-12
    s.close()


@pytest.mark.parametrize("p", [1, 2])
def test_solve_and_recover_match_oracle(p):
    mesh, prob, (tau, g, H, f), ru, rh = _case(p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-13, max_iter=2000)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-13
    for a, b in ((lam, lam0.reshape(lam.shape)), (u, u0), (h, h0)):
        assert _rel(a, b) <= 1e-10
    s.close()
    s8 = _solver(mesh, p, tau, g, H, f, rtol=1e-8, max_iter=2000, n_coarse=20)
    _, info8 = s8.solve(ru, rh)
    S = prob.trace_operator()
    pc = LFTwoLevelPreconditioner(prob, S, coarse="chebyshev", n_coarse=20, cheb_c=s8.chebyshev(coarse=True)[0])
    _, info0 = gmres(lambda v: S @ v, prob.condensed_rhs(ru, rh), pc, restart=30, rtol=1e-8, maxiter=2000)
    assert abs(info8["iters"] - info0["iters"]) <= 1, (info8["iters"], info0["iters"])
    s8.close()


def test_out_of_scope_configurations_are_rejected():
    from paper_2004_09389_gb300 import HDGSolver, HDGError, HDG_MIXED_FP32
    mesh, prob, (tau, g, H, f), _, _ = _case(1)
    for kw in (dict(precision=HDG_MIXED_FP32), dict(coarse_mode=2), dict(n_coarse=0)):
        with pytest.raises(HDGError):
            HDGSolver(mesh, 1, tau, g, H, f_vertex=f, flux=1, **kw)
    with pytest.raises(HDGError):
        HDGSolver(mesh, 3, tau, g, H, f_vertex=f, flux=1)
    sph = I.sphere_hierarchy(1, 1.0, r_coarsest=0)
    with pytest.raises(HDGError):
        HDGSolver(sph, 1, 0.1, 1.0, 1.0, flux=1)
