"""Mixed-precision condensation on the GPU (handles in HDG_MIXED_FP32 /
HDG_MIXED_BF16): A_K inverted in FP32, X = A_K^-1 [B_K | Mass_K] refined twice
with two-float residuals, S_K = Mt_K + C_K X_B and W_K = C_K R_M in two-float
arithmetic (Sec. 4.2 step 1 and Eq. schur_system, the local factorisation
in low precision recovered by refinement).

* Per-cell S_K equal the oracle's to 1e-12 of max |S_K| (two-float
  resolution), flat and sphere, p = 1..4.
* The trace operator applied to a vector equals the oracle's to 1e-12.
* A mixed solve followed by the recovery reaches the oracle's direct solution:
  lambda, u and h to 1e-9 at rtol 1e-11 (the recovery and the condensed
  right-hand side use W_K, X_B and R_M from this kernel).
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem

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


def _case(kind, p):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    tau = 8 * mesh.h / np.sqrt(g * H)
    return mesh, g, H, f, tau, HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f, tau_s=0.5)


@pytest.mark.parametrize("kind", ["flat", "sphere"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cell_schur_and_operator(kind, p):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, g, H, f, tau, prob = _case(kind, p)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=1, tau_s=0.5)
    S = s.cell_schur()
    S0 = np.stack([prob.cell_schur(K) for K in range(prob.N)])
    assert np.abs(S - S0).max() <= 1e-12 * np.abs(S0).max()
    x = np.random.default_rng(3).standard_normal(prob.n_trace)
    y = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.trace_apply_dev(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy(), prob.trace_operator() @ x) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p,precision", [("flat", 3, 1), ("sphere", 2, 1), ("flat", 2, 2)])
def test_mixed_solve_and_recovery(kind, p, precision):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, g, H, f, tau, prob = _case(kind, p)
    rng = np.random.default_rng(5)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=precision, rtol=1e-11, tau_s=0.5)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-11
    for a, b in ((lam, lam0.reshape(lam.shape)), (u, u0), (h, h0)):
        assert _rel(a, b) <= 1e-9
    s.close()
