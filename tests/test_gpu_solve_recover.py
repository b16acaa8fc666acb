"""Steps 1-3 with host buffers in one call (hdg_solve_recover, Sec. 4.2).

The one call runs the same kernels in the same order as hdg_solve followed by
hdg_recover with NULL lambda and right-hand sides, with one stream
synchronisation instead of two: lambda, u and h must be bit-identical to the
two calls', for mixed and FP64 handles, with pageable and page-locked host
buffers, and against the oracle's direct solve; an iteration limit returns
HDG_ENOCONV with the last iterate recovered, as the two calls do.
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


def _case(kind, p, seed=11):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(seed)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    return mesh, prob, (tau, g, H, f), ru, rh


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("kind,p,prec", [("flat", 2, 1), ("sphere", 3, 1), ("flat", 3, 0), ("sphere", 2, 0)])
@pytest.mark.parametrize("pinned", [False, True])
def test_one_call_matches_two_calls_and_oracle(kind, p, prec, pinned):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-10, precision=prec)
    if pinned:
        ru = torch.from_numpy(ru).pin_memory().numpy()
        rh = torch.from_numpy(rh).pin_memory().numpy()
    lam2, info2 = s.solve(ru, rh)
    u2, h2 = s.recover()
    lam1, u1, h1, info1 = s.solve_recover(ru, rh)
    assert info1["iters"] == info2["iters"] and info1["true_rel_res"] == info2["true_rel_res"]
    assert np.array_equal(lam1, lam2) and np.array_equal(u1, u2) and np.array_equal(h1, h2)
    # rtol 1e-10 bounds the error by kappa * 1e-10; kappa < 100 on these meshes
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert _rel(lam1, lam0.reshape(lam1.shape)) <= 1e-8
    assert _rel(u1, u0) <= 1e-8 and _rel(h1, h0) <= 1e-8
    s.close()


def test_iteration_limit_recovers_the_last_iterate():
    from paper_2004_09389_gb300 import HDGSolver
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = HDGSolver(mesh, 2, tau, g, H, f_vertex=f, rtol=1e-12, precision=0, max_iter=3)
    lam2, info2 = s.solve(ru, rh, allow_fail=True)
    u2, h2 = s.recover()
    lam1, u1, h1, info1 = s.solve_recover(ru, rh, allow_fail=True)
    assert info1["status"] == info2["status"] != 0
    assert np.array_equal(lam1, lam2) and np.array_equal(u1, u2) and np.array_equal(h1, h2)
    s.close()
