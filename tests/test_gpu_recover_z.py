"""Step 3 of a mixed-precision solve from what its step 1 kept (Sec. 4.2 steps 1
and 3, Eq. reconstruct_solution).

A two-float handle's solve forms z_K = A_K^-1 M_K r_K per cell in step 1 (and
the cell rows C_K z_K of the condensed right-hand side from the cell geometry);
hdg_recover_dev with NULL right-hand sides then forms q_K = z_K - A_K^-1 B_K
lambda_K without reading r or A_K^-1 M_K again.

* the two recovery routes (kept z_K, explicit r through A_K^-1 M_K) agree to
  1e-12 relative (two-float arithmetic, about 2^-46 per product, sums of at most
  3(p+1)(p+2)/2 + 3(p+1) terms), on flat and sphere meshes, every degree;
* the solve's lambda, u and h against the oracle's direct solve (1e-8 at rtol
  1e-10, as in the mixed-precision parity test): a wrong C_K z_K in step 1
  would move lambda;
* the state rules: one NULL right-hand side is HDG_EINVAL, and after the
  operator changes (hdg_set_tau) nothing is kept until the next solve;
* keep_rhs = 0 (step 1 from the stored C_K A_K^-1 M_K, nothing kept) solves to
  the same lambda and refuses a recovery with NULL right-hand sides.
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


def _case(kind, p, seed=3):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)       # 288 cells: 9 tiles of 32, full
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)            # 320 cells
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(seed)
    ru = rng.standard_normal((mesh.n_cells, 2, prob.np))
    rh = rng.standard_normal((mesh.n_cells, prob.np))
    return mesh, prob, (tau, g, H, f), ru, rh


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 2), ("flat", 3), ("flat", 4), ("sphere", 2),
                                    ("sphere", 3)])
def test_recovery_from_kept_z_matches_explicit_and_oracle(kind, p):
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-10, precision=HDG_MIXED_FP32)
    ru_d, rh_d = _dev(ru), _dev(rh)
    lam = torch.zeros((s.n_facets, p + 1), dtype=torch.float64, device="cuda")
    u_z = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
    h_z = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
    u_r, h_r = torch.empty_like(u_z), torch.empty_like(h_z)
    info = s.solve_dev(ru_d, rh_d, lam)
    s.recover_dev(None, None, None, u_z, h_z)          # from the kept z_K
    s.recover_dev(ru_d, rh_d, None, u_r, h_r)          # from r through A_K^-1 M_K
    torch.cuda.synchronize()
    assert info["true_rel_res"] <= 1e-10
    assert _rel(u_z.cpu().numpy(), u_r.cpu().numpy()) <= 1e-12
    assert _rel(h_z.cpu().numpy(), h_r.cpu().numpy()) <= 1e-12
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert _rel(lam.cpu().numpy(), lam0.reshape(lam.shape)) <= 1e-8
    assert _rel(u_z.cpu().numpy(), u0) <= 1e-8
    assert _rel(h_z.cpu().numpy(), h0) <= 1e-8
    s.close()


def test_null_right_hand_side_rules():
    from paper_2004_09389_gb300 import HDGSolver, HDGError, HDG_MIXED_FP32
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = HDGSolver(mesh, 2, tau, g, H, f_vertex=f, rtol=1e-10, precision=HDG_MIXED_FP32)
    ru_d, rh_d = _dev(ru), _dev(rh)
    lam = torch.zeros((s.n_facets, 3), dtype=torch.float64, device="cuda")
    u = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
    h = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError):
        s.recover_dev(None, None, None, u, h)          # no solve yet: nothing kept
    s.solve_dev(ru_d, rh_d, lam)
    with pytest.raises(HDGError):
        s.recover_dev(ru_d, None, None, u, h)          # one NULL right-hand side
    s.recover_dev(None, None, None, u, h)
    torch.cuda.synchronize()
    u_first = u.cpu().numpy().copy()
    s.set_tau(tau * 0.5)                                # the operator changes: z_K is stale
    with pytest.raises(HDGError):
        s.recover_dev(None, None, None, u, h)
    s.solve_dev(ru_d, rh_d, lam)                        # a new solve keeps a new z_K
    s.recover_dev(None, None, None, u, h)
    torch.cuda.synchronize()
    prob2 = HDGProblem(mesh, 2, tau=tau * 0.5, g=g, H=H, f_vertex=f)
    (u0, _), _ = prob2.solve_condensed(ru, rh)
    assert _rel(u.cpu().numpy(), u0) <= 1e-8
    assert _rel(u_first, u0) > 1e-6                     # the first recovery belonged to the old tau
    s.close()


def test_keep_rhs_off_keeps_nothing_and_solves_the_same():
    """keep_rhs = 0: step 1 reads C_K A_K^-1 M_K and keeps nothing for the
    recovery; the solve reaches the same lambda (both to rtol 1e-10)."""
    from paper_2004_09389_gb300 import HDGSolver, HDGError, HDG_MIXED_FP32
    mesh, prob, (tau, g, H, f), ru, rh = _case("sphere", 3)
    ru_d, rh_d = _dev(ru), _dev(rh)
    lams = []
    for keep in (1, 0):
        s = HDGSolver(mesh, 3, tau, g, H, f_vertex=f, rtol=1e-10, precision=HDG_MIXED_FP32, keep_rhs=keep)
        lam = torch.zeros((s.n_facets, 4), dtype=torch.float64, device="cuda")
        u = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
        h = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
        info = s.solve_dev(ru_d, rh_d, lam)
        assert info["true_rel_res"] <= 1e-10
        if keep:
            s.recover_dev(None, None, None, u, h)
        else:
            with pytest.raises(HDGError):
                s.recover_dev(None, None, None, u, h)
            s.recover_dev(ru_d, rh_d, None, u, h)
        torch.cuda.synchronize()
        (u0, _), _ = prob.solve_condensed(ru, rh)
        assert _rel(u.cpu().numpy(), u0) <= 1e-8
        lams.append(lam.cpu().numpy())
        s.close()
    assert _rel(lams[1], lams[0]) <= 1e-9
