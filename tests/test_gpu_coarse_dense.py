"""Large coarsest P1 levels on the GPU: when the single-CTA coarse cycle would
hold only the coarsest level and that level has more than 256 vertices, the
coarse problem's last level is solved exactly by a multi-CTA product with its
FP64 inverse, which the condensation computes by the multi-launch Gauss-Jordan
elimination (Alg. twolevel_vcycle line 4 with the P1 hierarchy truncated at
the coarsest level).

* One preconditioner application equals the oracle's on the same hierarchy
  (1e-12 FP64, 1e-5 FP32), flat (1024-vertex coarsest) and sphere (642).
* Solves reach the oracle's direct solution (1e-10 at rtol 1e-12, FP64 and
  the mixed mode), with the oracle's iteration count within one.
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


def _case(kind):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(64, n_coarsest=32)      # P1 levels 4096, 1024
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(4, 1.0, r_coarsest=3)             # P1 levels 2562, 642
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    return mesh, g, H, f


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("sphere", 2)])
def test_precond_matches_oracle(kind, p):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, g, H, f = _case(kind)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), coarse="gmg")
    v = np.random.default_rng(17).standard_normal(prob.n_trace)
    z0 = pc(v)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=1)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    z32 = torch.empty(prob.n_trace, dtype=torch.float32, device="cuda")
    s.precond_apply_dev(torch.from_numpy(v).cuda(), z)
    s.precond_apply32_dev(torch.from_numpy(v.astype(np.float32)).cuda(), z32)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), z0) <= 1e-12
    assert _rel(z32.cpu().numpy().astype(np.float64), z0) <= 1e-5
    s.close()


@pytest.mark.parametrize("kind,p,precision", [("flat", 2, 0), ("sphere", 3, 0), ("flat", 3, 1)])
def test_solve_matches_oracle(kind, p, precision):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, g, H, f = _case(kind)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(19)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-12, precision=precision)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-12
    for a, b in ((lam, lam0.reshape(lam.shape)), (u, u0), (h, h0)):
        assert _rel(a, b) <= 1e-10
    s.close()
    if precision == 0:
        s8 = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-8, precision=0)
        _, info8 = s8.solve(ru, rh)
        S = prob.trace_operator()
        pc = TwoLevelPreconditioner(prob, mesh, S, coarse="gmg")
        _, info0 = gmres(lambda v: S @ v, prob.condensed_rhs(ru, rh), pc, restart=30, rtol=1e-8)
        assert abs(info8["iters"] - info0["iters"]) <= 1
        s8.close()
