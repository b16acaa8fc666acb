"""Merged batched solves (GPU): one host thread, the launches of all
problems merged into multi-problem kernels, one CUDA graph per wave.

* Every problem's result is bit-identical to the same handle's hdg_solve_dev
  run alone, with the same iteration count, for a mix of meshes, degrees,
  tau, smoothers and both mixed precisions; a second batched call (every
  wave replayed from its kept graph) again gives the same bits.
* The batched results match the oracle's direct solve.
* Launches per wave do not grow with the number of problems: k problems of
  the same structure in one group take exactly the merged launches of one,
  carrying k times the per-problem launches.
* Handles that the merged path does not run are refused.
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
    # kind, size, p, tau scale, smoother, precision (1: HDG_MIXED_FP32, 2: HDG_MIXED_BF16)
    specs = [("flat", 8, 1, 1.0, 0, 1), ("flat", 12, 2, 2.0, 0, 1), ("sphere", 2, 2, 1.0, 1, 1),
             ("flat", 16, 3, 4.0, 0, 1), ("sphere", 1, 3, 2.0, 0, 2), ("flat", 24, 2, 2.0, 1, 1),
             ("sphere", 3, 1, 2.0, 0, 1), ("flat", 12, 3, 1.0, 0, 2)]
    for k, (kind, size, p, tscale, sm, prec) in enumerate(specs):
        if kind == "flat":
            mesh = I.periodic_square_hierarchy(size, n_coarsest=3)
            f = I.coriolis_flat(mesh, 1.0)
        else:
            mesh = I.sphere_hierarchy(size, 1.0, r_coarsest=0)
            f = I.coriolis_sphere(mesh, 0.5)
        tau = 4.0 * tscale * mesh.h
        rng = np.random.default_rng(300 + k)
        n_p = (p + 1) * (p + 2) // 2
        ru = rng.standard_normal((mesh.n_cells, 2, n_p))
        rh = rng.standard_normal((mesh.n_cells, n_p))
        out.append(dict(mesh=mesh, p=p, tau=tau, f=f, ru=ru, rh=rh, smoother=sm, precision=prec))
    return out


def _solver(x, rtol=1e-10):
    from paper_2004_09389_gb300 import HDGSolver
    return HDGSolver(x["mesh"], x["p"], x["tau"], 1.0, 1.0, f_vertex=x["f"], rtol=rtol,
                     precision=x["precision"], smoother=x["smoother"])


def test_merged_batch_bit_identical_and_oracle():
    from paper_2004_09389_gb300 import MergedBatch
    probs = _problems()
    solvers = [_solver(x) for x in probs]
    ru = [torch.from_numpy(x["ru"]).cuda() for x in probs]
    rh = [torch.from_numpy(x["rh"]).cuda() for x in probs]
    single, single_info = [], []
    for s, a, b in zip(solvers, ru, rh):
        lam = torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda")
        single_info.append(s.solve_dev(a, b, lam))
        single.append(lam)
    torch.cuda.synchronize()
    batch = MergedBatch(solvers)
    # the same output buffers both times: the waves (whose records carry
    # every argument, these pointers included) recur exactly
    lam = [torch.empty((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
    # host buffers: the same bits through the staging copies
    lam_h, infos_h = batch.solve([x["ru"] for x in probs], [x["rh"] for x in probs])
    for i, (l, l0, info, info0) in enumerate(zip(lam_h, single, infos_h, single_info)):
        assert np.array_equal(l, l0.cpu().numpy()), i
        assert info["iters"] == info0["iters"], i
    st = []
    for rep in range(2):
        for l in lam:
            l.fill_(float("nan"))
        infos = batch.solve_dev(ru, rh, lam)
        st.append(batch.stats())
        for i, (l, l0, info, info0) in enumerate(zip(lam, single, infos, single_info)):
            assert torch.equal(l, l0), (rep, i)
            assert info["iters"] == info0["iters"], (rep, i)
            assert info["true_rel_res"] == info0["true_rel_res"], (rep, i)
            assert info["true_rel_res"] <= 1e-10
    # the second device call replays kept graphs only (a wave can also recur
    # within one call, e.g. the first Arnoldi step of every refinement pass)
    assert st[0]["builds"] > 0 and st[1]["builds"] == st[0]["builds"]
    assert st[1]["replays"] - st[0]["replays"] == st[1]["waves"] - st[0]["waves"] > 0
    assert st[1]["records"] > st[1]["launches"]       # launches of different problems were merged
    for x, l in zip(probs, lam):
        prob = HDGProblem(x["mesh"], x["p"], tau=x["tau"], g=1.0, H=1.0, f_vertex=x["f"])
        _, lam0 = prob.solve_condensed(x["ru"], x["rh"])
        lb = l.cpu().numpy().ravel()
        tol = 1e-6 if x["precision"] == 2 else 1e-7
        assert np.linalg.norm(lb - lam0) <= tol * np.linalg.norm(lam0)
    batch.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("k", [3, 12])
def test_merged_launches_do_not_grow_with_problems(k, monkeypatch):
    from paper_2004_09389_gb300 import MergedBatch
    monkeypatch.setenv("HDG_BATCH_GROUPS", "1")     # all problems in one group
    x = _problems()[3]
    counts = {}
    for n in (1, k):
        solvers = [_solver(x) for _ in range(n)]
        ru = [torch.from_numpy(x["ru"]).cuda() for _ in range(n)]
        rh = [torch.from_numpy(x["rh"]).cuda() for _ in range(n)]
        lam = [torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
        batch = MergedBatch(solvers)
        infos = batch.solve_dev(ru, rh, lam)
        counts[n] = batch.stats()
        for l in lam[1:]:
            assert torch.equal(l, lam[0])
        assert len({i["iters"] for i in infos}) == 1
        batch.close()
        for s in solvers:
            s.close()
    one, many = counts[1], counts[k]
    assert many["waves"] == one["waves"]
    assert many["launches"] == one["launches"]
    assert many["records"] == k * one["records"]


def test_merged_batch_refuses_unsupported_handles():
    from paper_2004_09389_gb300 import HDGError, HDGSolver, MergedBatch
    x = _problems()[0]
    s64 = HDGSolver(x["mesh"], x["p"], x["tau"], 1.0, 1.0, f_vertex=x["f"], precision=0)
    with pytest.raises(HDGError, match="HDG_MIXED_FP32"):
        MergedBatch([s64])
    s = _solver(x)
    with pytest.raises(HDGError, match="same handle twice"):
        MergedBatch([s, s])
    b = MergedBatch([s])
    s.profile_enable(True)
    t = torch.from_numpy(x["ru"]).cuda(), torch.from_numpy(x["rh"]).cuda()
    lam = torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError, match="kernel timing"):
        b.solve_dev([t[0]], [t[1]], [lam])
    s.profile_enable(False)
    info = b.solve_dev([t[0]], [t[1]], [lam])[0]
    assert info["true_rel_res"] <= 1e-10
    b.close()
    s.close()
    s64.close()


def test_merged_batch_reports_failing_problems():
    """A problem that stops on its iteration limit and one with a NaN in its
    right-hand side report HDG_ENOCONV / HDG_ENAN through their info entries;
    the batch returns the first failure in problem order, and the other
    problems finish exactly as their own solves do."""
    from paper_2004_09389_gb300 import HDGError, HDGSolver, MergedBatch
    from paper_2004_09389_gb300 import _lib as L
    probs = _problems()[:4]
    solvers = [_solver(x) for x in probs]
    probs[1] = dict(probs[1])
    solvers[1].close()
    x1 = probs[1]
    solvers[1] = HDGSolver(x1["mesh"], x1["p"], x1["tau"], 1.0, 1.0, f_vertex=x1["f"], rtol=1e-10,
                           precision=x1["precision"], smoother=x1["smoother"], max_iter=2)
    ru = [torch.from_numpy(x["ru"]).cuda() for x in probs]
    rh = [torch.from_numpy(x["rh"]).cuda() for x in probs]
    rh[3] = rh[3].clone()
    rh[3][0, 0] = float("nan")
    single = []
    for k in (0, 2):
        lam = torch.zeros((solvers[k].n_facets, solvers[k].p + 1), dtype=torch.float64, device="cuda")
        solvers[k].solve_dev(ru[k], rh[k], lam)
        single.append(lam)
    lam = [torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
    b = MergedBatch(solvers)
    with pytest.raises(HDGError) as ei:
        b.solve_dev(ru, rh, lam)
    assert ei.value.code == L.HDG_ENOCONV and "batch entry 1" in str(ei.value)
    infos = b.solve_dev(ru, rh, lam, allow_fail=True)
    assert infos[1]["status"] == L.HDG_ENOCONV
    assert infos[3]["status"] == L.HDG_ENAN
    assert infos[0]["status"] == 0 and infos[2]["status"] == 0
    assert torch.equal(lam[0], single[0]) and torch.equal(lam[2], single[1])
    b.close()
    for s in solvers:
        s.close()
