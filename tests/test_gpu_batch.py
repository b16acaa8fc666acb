"""Batched solves and the launch-shape autotuner (GPU).

* hdg_solve_batch_dev runs independent problems of uneven size, degree and
  tau concurrently; every result is bit-identical to the same handle's solve
  run alone (same kernels, same launch shapes, deterministic reductions) and
  matches the oracle's direct solve.
* hdg_autotune changes launch shapes only: the solution agrees with the
  untuned one to 1e-10 relative with the same iteration count.
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


def _problems():
    out = []
    specs = [("flat", 8, 1, 1.0), ("flat", 12, 2, 2.0), ("sphere", 2, 2, 1.0), ("flat", 16, 3, 4.0),
             ("sphere", 1, 3, 2.0), ("flat", 6, 4, 1.0)]
    for k, (kind, size, p, tscale) in enumerate(specs):
        if kind == "flat":
            mesh = I.periodic_square_hierarchy(size, n_coarsest=3)
            f = I.coriolis_flat(mesh, 1.0)
        else:
            mesh = I.sphere_hierarchy(size, 1.0, r_coarsest=0)
            f = I.coriolis_sphere(mesh, 0.5)
        tau = 4.0 * tscale * mesh.h
        rng = np.random.default_rng(100 + k)
        n_p = (p + 1) * (p + 2) // 2
        ru = rng.standard_normal((mesh.n_cells, 2, n_p))
        rh = rng.standard_normal((mesh.n_cells, n_p))
        out.append((mesh, p, tau, f, ru, rh))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_and_oracle(precision):
    from paper_2004_09389_gb300 import HDGSolver, solve_batch_dev
    probs = _problems()
    solvers = [HDGSolver(m, p, tau, 1.0, 1.0, f_vertex=f, rtol=1e-11, precision=precision)
               for (m, p, tau, f, _, _) in probs]
    ru = [torch.from_numpy(x[4]).cuda() for x in probs]
    rh = [torch.from_numpy(x[5]).cuda() for x in probs]
    lam = [torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
    torch.cuda.synchronize()
    infos = solve_batch_dev(solvers, ru, rh, lam, n_threads=4)
    torch.cuda.synchronize()
    for s, x, l, info in zip(solvers, probs, lam, infos):
        mesh, p, tau, f, ru_h, rh_h = x
        assert info["true_rel_res"] <= 1e-11
        single = torch.zeros_like(l)
        s.solve_dev(torch.from_numpy(ru_h).cuda(), torch.from_numpy(rh_h).cuda(), single)
        torch.cuda.synchronize()
        assert torch.equal(single, l)
        prob = HDGProblem(mesh, p, tau=tau, g=1.0, H=1.0, f_vertex=f)
        _, lam0 = prob.solve_condensed(ru_h, rh_h)
        lb = l.cpu().numpy().ravel()
        assert np.linalg.norm(lb - lam0) <= 1e-8 * np.linalg.norm(lam0)
        s.close()


def test_batch_rejects_shared_handles():
    from paper_2004_09389_gb300 import HDGSolver, solve_batch_dev, HDGError
    mesh, p, tau, f, ru, rh = _problems()[0]
    s = HDGSolver(mesh, p, tau, 1.0, 1.0, f_vertex=f)
    t = torch.from_numpy(ru).cuda(), torch.from_numpy(rh).cuda()
    lam = torch.zeros((s.n_facets, p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError):
        solve_batch_dev([s, s], [t[0], t[0]], [t[1], t[1]], [lam, lam])
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_the_solution(precision):
    from paper_2004_09389_gb300 import HDGSolver
    mesh = I.periodic_square_hierarchy(64, n_coarsest=4)
    p = 2
    tau = 8 * mesh.h
    f = I.coriolis_flat(mesh, 1.0)
    rng = np.random.default_rng(5)
    ru = rng.standard_normal((mesh.n_cells, 2, 6))
    rh = rng.standard_normal((mesh.n_cells, 6))
    s = HDGSolver(mesh, p, tau, 1.0, 1.0, f_vertex=f, rtol=1e-10, precision=precision)
    lam0, info0 = s.solve(ru, rh)
    choice = s.autotune()
    assert choice[0] in (64, 128, 256) and choice[1] in (152, 304, 608, 1216) and choice[2] > 0
    lam1, info1 = s.solve(ru, rh)
    assert info1["true_rel_res"] <= 1e-10
    assert abs(info1["iters"] - info0["iters"]) <= 1
    assert np.linalg.norm(lam1 - lam0) <= 1e-9 * np.linalg.norm(lam0)
    s.close()
