"""Parity at the benchmark's full sizes, in the benchmark's launch configuration.

Workloads: flat periodic 256 x 256 x 2 (131,072 triangles), p = 3, acoustic
Courant 8, g = 9.81, H = 1e3, f = 1e-4, k^-3 Gaussian right-hand sides; and
the icosahedral sphere r = 6 (81,920 triangles, radius 6.371e6 m, f =
2 Omega sin(latitude), p = 3, Courant 8, spherical-harmonic right-hand sides).
The oracle cannot solve these sizes in seconds, so it checks sampled outputs
one by one (trace-operator rows, condensed right-hand side, recovered cells)
and the solve is checked through properties that hold at any size: the true
relative residual of the returned lambda, and discrete mass conservation up
to the bound the residual implies.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=["flat", "sphere"])
def setup(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build, HDGSolver, HDG_FP64, HDG_MIXED_FP32
    from oracle.hdg import HDGProblem, MeshData, local_coordinates
    import bench
    build.build()
    p = 3
    wl = bench.make_workload(request.param, True, p, 8.0, 0)
    mesh, tau, f, ru, rh, g, H = wl["mesh"], wl["tau"], wl["f"], wl["ru"], wl["rh"], wl["g"], wl["H"]
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f, lazy=True)
    s64 = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=HDG_FP64, rtol=1e-8)
    s32 = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=HDG_MIXED_FP32, rtol=1e-8)
    X = local_coordinates(MeshData.of(mesh))
    detJ = np.abs((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1])
                  - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1]))
    yield dict(mesh=mesh, tau=tau, f=f, ru=ru, rh=rh, prob=prob, s64=s64, s32=s32, p=p, detJ=detJ)
    s64.close()
    s32.close()


def _samples(n, k=64, seed=0):
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[0, n - 1, rng.integers(0, n, k)])


def test_facets_match_oracle_numbering(setup):
    fo, fl, fv = setup["s64"].facets()
    prob = setup["prob"]
    assert (fo == prob.facet_of).all() and (fl == prob.flip).all() and (fv == prob.facet_verts).all()


def test_trace_apply_sampled_rows(setup):
    s, prob = setup["s64"], setup["prob"]
    x = np.random.default_rng(1).standard_normal(prob.n_trace)
    y = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.trace_apply_dev(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    y = y.cpu().numpy().reshape(prob.n_facets, -1)
    fac = _samples(prob.n_facets)
    y0 = prob.facet_rows(fac, x)
    assert np.abs(y[fac] - y0).max() <= 1e-12 * np.abs(y0).max()


def test_condensed_rhs_sampled(setup):
    s, prob = setup["s64"], setup["prob"]
    g = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.condensed_rhs_dev(torch.from_numpy(setup["ru"]).cuda(), torch.from_numpy(setup["rh"]).cuda(), g)
    torch.cuda.synchronize()
    g = g.cpu().numpy().reshape(prob.n_facets, -1)
    fac = _samples(prob.n_facets, seed=2)
    g0 = prob.facet_rhs(fac, setup["ru"], setup["rh"])
    assert np.abs(g[fac] - g0).max() <= 1e-12 * np.abs(g0).max()


@pytest.mark.parametrize("arm", ["s64", "s32"])
def test_solve_properties_and_sampled_recovery(setup, arm):
    s, prob = setup[arm], setup["prob"]
    ru, rh = setup["ru"], setup["rh"]
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    assert info["true_rel_res"] <= 1e-8
    # independent residual check with the (sample-verified) FP64 operator
    ru_d, rh_d = torch.from_numpy(ru).cuda(), torch.from_numpy(rh).cuda()
    g = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    setup["s64"].condensed_rhs_dev(ru_d, rh_d, g)
    Sl = torch.empty_like(g)
    setup["s64"].trace_apply_dev(torch.from_numpy(lam).cuda().reshape(-1), Sl)
    torch.cuda.synchronize()
    res = (g - Sl).cpu().numpy()
    rel = np.linalg.norm(res) / np.linalg.norm(g.cpu().numpy())
    assert rel <= 1.5e-8
    # mass conservation: int h - int r_h = -tau * sum of the facet residuals (mu = 1);
    # int_K phi_i = |det J_K| times its reference-triangle integral
    prob_w = np.asarray(__import__("oracle.reference", fromlist=["x"]).reference_matrices(setup["p"])["M"]).sum(0)
    dj = setup["detJ"]
    mass_h = (dj * (h @ prob_w)).sum()
    mass_r = (dj * (rh @ prob_w)).sum()
    assert abs((mass_h - mass_r) + setup["tau"] * res.sum()) <= 1e-9 * (dj * np.abs(rh @ prob_w)).sum()
    # sampled cells recovered exactly from this lambda
    cells = _samples(prob.N, seed=3)
    q0 = prob.local_cells(cells, ru, rh, lam.reshape(-1))
    q = np.concatenate([u[cells, 0], u[cells, 1], h[cells]], axis=1)
    assert np.abs(q - q0).max() <= 1e-11 * np.abs(q0).max()

