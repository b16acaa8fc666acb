"""Galerkin coarse operators on the GPU (coarse_mode = 2: pi^T S pi on the fine
P1 level and P^T A P below it, the alternative of the Sec. 4.4 footnote)
against the oracle's Galerkin hierarchy.

* One preconditioner application equals the oracle's with the same coarse
  operators (1e-12), flat and sphere, p = 1 and 3, with the coarse levels in
  the single-CTA cycle; with them in the multi-block (patch-fused and
  unfused) kernels on a mixed-precision handle (two-float condensation),
  1e-11 in FP64 and 1e-5 in FP32.
* Solves reach the oracle's direct solution (1e-10 at rtol 1e-13), with the
  oracle's iteration count within one; also together with the Chebyshev
  smoother.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem
from oracle.solver import TwoLevelPreconditioner, gmres

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


def _case(kind, big=False):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(24 if big else 12, n_coarsest=3)
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(3 if big else 2, 1.0, r_coarsest=0)
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    return mesh, g, H, f


def _solver(mesh, p, tau, g, H, f, **kw):
    from paper_2004_09389_gb300 import HDGSolver
    return HDGSolver(mesh, p, tau, g, H, f_vertex=f, coarse_mode=2, **kw)


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("sphere", 1), ("sphere", 3)])
def test_precond_matches_oracle(kind, p):
    mesh, g, H, f = _case(kind)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    s = _solver(mesh, p, tau, g, H, f)
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), coarse="gmg", coarse_mode="galerkin")
    v = np.random.default_rng(7).standard_normal(prob.n_trace)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.precond_apply_dev(torch.from_numpy(v).cuda(), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), pc(v)) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_precond_multi_block_levels_match_oracle(kind, monkeypatch):
    mesh, g, H, f = _case(kind, big=True)
    p = 1
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), coarse="gmg", coarse_mode="galerkin")
    v = np.random.default_rng(8).standard_normal(prob.n_trace)
    z0 = pc(v)
    monkeypatch.setenv("HDG_TAIL_MAX_VERTICES", "16")
    for fused in ("1", "0"):
        monkeypatch.setenv("HDG_P1_FUSED", fused)
        s = _solver(mesh, p, tau, g, H, f, precision=1)
        z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
        z32 = torch.empty(prob.n_trace, dtype=torch.float32, device="cuda")
        s.precond_apply_dev(torch.from_numpy(v).cuda(), z)
        s.precond_apply32_dev(torch.from_numpy(v.astype(np.float32)).cuda(), z32)
        torch.cuda.synchronize()
        # a mixed-precision handle condenses in two-float arithmetic (about
        # 2^-48 per S_K entry), and the Galerkin coarse operator sums S_K
        # entries with cancellation: its FP64 application agrees to 1e-11
        assert _rel(z.cpu().numpy(), z0) <= 1e-11, fused
        assert _rel(z32.cpu().numpy().astype(np.float64), z0) <= 1e-5, fused
        s.close()


@pytest.mark.parametrize("kind,p,smoother", [("flat", 2, 0), ("sphere", 3, 0), ("sphere", 2, 1)])
def test_solve_matches_oracle(kind, p, smoother):
    mesh, g, H, f = _case(kind)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(9)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-13, smoother=smoother)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-13
    for a, b in ((lam, lam0.reshape(lam.shape)), (u, u0), (h, h0)):
        assert _rel(a, b) <= 1e-10
    s.close()
    s8 = _solver(mesh, p, tau, g, H, f, rtol=1e-8, smoother=smoother)
    _, info8 = s8.solve(ru, rh)
    S = prob.trace_operator()
    kw = dict(smoother="chebyshev", cheb=s8.chebyshev()[0]) if smoother else {}
    pc = TwoLevelPreconditioner(prob, mesh, S, coarse="gmg", coarse_mode="galerkin", **kw)
    _, info0 = gmres(lambda v: S @ v, prob.condensed_rhs(ru, rh), pc, restart=30, rtol=1e-8)
    assert abs(info8["iters"] - info0["iters"]) <= 1
    s8.close()
