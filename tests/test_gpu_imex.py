"""IMEX time stepping on the GPU (hdg_imex_*, through the C ABI) against the
IMEX oracle (oracle/imex.py): Sec. 3.3 (Eq. theta_method, Eqs. IMEX_HDG_I and
IMEX_HDG_II) with the tableaux of Sec. 5.1, Coriolis explicit as in the paper.

* The stage rates M^-1 N(q) and M^-1 L(q) of random states equal the oracle's
  -M^-1 C q and -M^-1 K0 q (standard upwind DG operator extracted from the
  assembly) to 1e-12 relative, flat and sphere, p = 1..4.
* One step of theta (1/2 and 1), ARS2(2,3,2), SSP2(3,2,2) and ARS3(4,4,3) from
  the same state, FP64 solves to rtol 1e-13, equals the oracle's step with
  direct stage solves to 1e-10 relative per field; mixed precision to 1e-7.
* Five ARS2 steps stay within 1e-10 of the oracle and conserve mass (the
  integral of h) to the stage solves' tolerance.
* Error paths: a handle with a Coriolis field in its implicit operator, an
  unknown scheme, dt <= 0, calls before hdg_imex_init.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle import imex

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build
    build.build()


def _case(kind, p):
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)         # 288 cells: several tiles, ragged tail
        g, H, f = 1.0, 1.0, I.coriolis_flat(mesh, 2.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)              # 320 cells
        g, H, f = 1.3, 0.7, I.coriolis_sphere(mesh, 1.5)
    return mesh, g, H, f


def _state(ops, seed):
    q = np.random.default_rng(seed).standard_normal((ops.N, 3, ops.np))
    q[:, 2, :] += 0.7
    return q


def _split(q):
    return np.ascontiguousarray(q[:, :2, :]), np.ascontiguousarray(q[:, 2, :])


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _solver(mesh, p, g, H, f, **kw):
    from paper_2004_09389_gb300 import HDGSolver
    s = HDGSolver(mesh, p, 0.1, g, H, f_vertex=None, condense=False, **kw)
    s.imex_init(f)
    return s


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 2), ("flat", 3), ("flat", 4), ("sphere", 2), ("sphere", 3)])
def test_stage_rates_match_oracle(kind, p):
    mesh, g, H, f = _case(kind, p)
    ops = imex.IMEXOperators(mesh, p, g, H, f)
    s = _solver(mesh, p, g, H, f)
    q = _state(ops, 3)
    u, h = _split(q)
    ud, hd = torch.from_numpy(u).cuda(), torch.from_numpy(h).cuda()
    nu, nh, lu, lh = (torch.empty_like(x) for x in (ud, hd, ud, hd))
    s.imex_rates_dev(ud, hd, nu, nh, lu, lh)
    torch.cuda.synchronize()
    n_ref = ops.mass_solve(-(ops.C @ q.ravel())).reshape(q.shape)
    l_ref = ops.mass_solve(-(ops.K0 @ q.ravel())).reshape(q.shape)
    assert _rel(lu.cpu().numpy(), l_ref[:, :2]) <= 1e-12
    assert _rel(lh.cpu().numpy(), l_ref[:, 2]) <= 1e-12
    assert _rel(nu.cpu().numpy(), n_ref[:, :2]) <= 1e-12
    assert np.abs(nh.cpu().numpy()).max() == 0.0
    s.close()


def _oracle_step(ops, q, dt, scheme, theta):
    if scheme == "theta":
        return imex.theta_step(ops, q.ravel(), dt, theta).reshape(q.shape)
    return imex.imex_rk_step(ops, q.ravel(), dt, scheme).reshape(q.shape)


@pytest.mark.parametrize("scheme,theta", [("theta", 0.5), ("theta", 1.0), ("ARS2", 0.0), ("SSP2", 0.0),
                                          ("ARS3", 0.0)])
@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 3)])
def test_one_step_matches_oracle(kind, p, scheme, theta):
    mesh, g, H, f = _case(kind, p)
    ops = imex.IMEXOperators(mesh, p, g, H, f)
    dt = 4 * mesh.h / np.sqrt(g * H)                # acoustic Courant number 4 per step
    q = _state(ops, 5)
    ref = _oracle_step(ops, q, dt, scheme, theta)
    s = _solver(mesh, p, g, H, f, rtol=1e-13)
    u, h = _split(q)
    ud, hd = torch.from_numpy(u).cuda(), torch.from_numpy(h).cuda()
    info = s.imex_step_dev(scheme, dt, ud, hd, theta=theta)
    assert info["status"] == 0 and info["iters"] > 0
    assert _rel(ud.cpu().numpy(), ref[:, :2]) <= 1e-10
    assert _rel(hd.cpu().numpy(), ref[:, 2]) <= 1e-10
    s.close()


def test_mixed_precision_step_matches_oracle():
    from paper_2004_09389_gb300 import HDG_MIXED_FP32
    mesh, g, H, f = _case("sphere", 2)
    ops = imex.IMEXOperators(mesh, 2, g, H, f)
    dt = 4 * mesh.h / np.sqrt(g * H)
    q = _state(ops, 6)
    ref = _oracle_step(ops, q, dt, "ARS2", 0.0)
    s = _solver(mesh, 2, g, H, f, rtol=1e-10, precision=HDG_MIXED_FP32)
    u, h = _split(q)
    ud, hd = torch.from_numpy(u).cuda(), torch.from_numpy(h).cuda()
    s.imex_step_dev("ARS2", dt, ud, hd)
    assert _rel(ud.cpu().numpy(), ref[:, :2]) <= 1e-7
    assert _rel(hd.cpu().numpy(), ref[:, 2]) <= 1e-7
    s.close()


def test_several_steps_match_oracle_and_conserve_mass():
    mesh, g, H, f = _case("flat", 2)
    ops = imex.IMEXOperators(mesh, 2, g, H, f)
    dt = 4 * mesh.h / np.sqrt(g * H)
    q = _state(ops, 7)
    s = _solver(mesh, 2, g, H, f, rtol=1e-13)
    u, h = _split(q)
    ud, hd = torch.from_numpy(u).cuda(), torch.from_numpy(h).cuda()
    mass0 = ops.integral_of_h(q.ravel())
    for _ in range(5):
        q = _oracle_step(ops, q, dt, "ARS2", 0.0)
        s.imex_step_dev("ARS2", dt, ud, hd)
    assert _rel(ud.cpu().numpy(), q[:, :2]) <= 1e-10
    assert _rel(hd.cpu().numpy(), q[:, 2]) <= 1e-10
    qg = np.concatenate([ud.cpu().numpy(), hd.cpu().numpy()[:, None, :]], axis=1)
    assert abs(ops.integral_of_h(qg.ravel()) - mass0) <= 1e-11 * abs(mass0)
    s.close()


def test_error_paths():
    from paper_2004_09389_gb300 import HDGSolver, HDGError
    mesh, g, H, f = _case("flat", 1)
    with_f = HDGSolver(mesh, 1, 0.1, g, H, f_vertex=f, condense=False)
    with pytest.raises(HDGError):
        with_f.imex_init(f)                       # the implicit operator must have no Coriolis term
    with_f.close()
    s = HDGSolver(mesh, 1, 0.1, g, H, condense=False)
    ud = torch.zeros((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
    hd = torch.zeros((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError):
        s.imex_step_dev("ARS2", 0.1, ud, hd)      # before hdg_imex_init
    s.imex_init(f)
    with pytest.raises(HDGError):
        s.imex_step_dev(7, 0.1, ud, hd)
    with pytest.raises(HDGError):
        s.imex_step_dev("ARS2", -0.1, ud, hd)
    with pytest.raises(HDGError):
        s.imex_step_dev("theta", 0.1, ud, hd, theta=0.0)
    s.close()
