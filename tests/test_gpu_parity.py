"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Tolerances (FP64 path): cell blocks, trace operator, right-hand side,
preconditioner and recovery agree to <= 1e-12 relative (same arithmetic up to
rounding order, operators of norm ~1); the end-to-end solve, run to a true
relative residual of 1e-13, agrees with the oracle's direct solve to <= 1e-10
relative in every field (lambda, u, h).  Mixed mode: see test_mixed_precision.
Integer data (facet numbering, orientation) must match exactly.
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


def _solver(mesh, p, tau, g, H, f, **kw):
    from paper_2004_09389_gb300 import HDGSolver
    return HDGSolver(mesh, p, tau, g, H, f_vertex=f, **kw)


def _case(kind, p, seed=0):
    """Small meshes spanning several 256-thread tiles with a ragged tail."""
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(12, n_coarsest=3)       # 288 cells, 432 facets
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)            # 320 cells, 480 facets
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


CASES = [("flat", 1), ("flat", 2), ("flat", 3), ("flat", 4), ("sphere", 1), ("sphere", 3)]


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_facet_numbering_matches_oracle(kind):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, 1)
    s = _solver(mesh, 1, tau, g, H, f, condense=False)
    fo, fl, fv = s.facets()
    assert (fo == prob.facet_of).all()
    assert (fl == prob.flip.astype(np.int32)).all()
    assert (fv == prob.facet_verts).all()
    s.close()


@pytest.mark.parametrize("kind,p", CASES)
def test_cell_schur_matches_oracle(kind, p):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f)
    S = s.cell_schur()
    S0 = np.stack([prob.cell_schur(K) for K in range(prob.N)])
    assert np.abs(S - S0).max() <= 1e-12 * np.abs(S0).max()
    s.close()


@pytest.mark.parametrize("kind,p", CASES)
def test_trace_apply_matches_oracle(kind, p):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f)
    x = np.random.default_rng(1).standard_normal(prob.n_trace)
    y0 = prob.trace_operator() @ x
    y = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.trace_apply_dev(_dev(x), y)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy(), y0) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p", CASES)
def test_condensed_rhs_matches_oracle(kind, p):
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f)
    g0 = prob.condensed_rhs(ru, rh)
    gd = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.condensed_rhs_dev(_dev(ru), _dev(rh), gd)
    torch.cuda.synchronize()
    assert _rel(gd.cpu().numpy(), g0) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("sphere", 2)])
@pytest.mark.parametrize("n_pre,n_post", [(2, 2), (0, 1), (1, 0), (3, 3)])
def test_precond_matches_oracle(kind, p, n_pre, n_post):
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, n_pre=n_pre, n_post=n_post)
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S, n_pre=n_pre, n_post=n_post, coarse="gmg")
    v = np.random.default_rng(2).standard_normal(prob.n_trace)
    z0 = pc(v)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.precond_apply_dev(_dev(v), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), z0) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_precond_printed_coarse_form_matches_oracle(kind):
    """coarse_mode = 1: the coarse operator exactly as printed (no rotation)."""
    mesh, prob, (tau, g, H, f), _, _ = _case(kind, 2)
    s = _solver(mesh, 2, tau, g, H, f, coarse_mode=1)
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), coarse="gmg", coarse_mode="rediscretised")
    v = np.random.default_rng(4).standard_normal(prob.n_trace)
    z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
    s.precond_apply_dev(_dev(v), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy(), pc(v)) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p", CASES)
@pytest.mark.parametrize("reorth", [0, 1])
def test_solve_and_recover_match_oracle(kind, p, reorth):
    """One classical Gram-Schmidt pass (reorth 0, the default) and CGS2
    (reorth 1) both reach the oracle's solution."""
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-13, reorth=reorth)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-13
    assert _rel(lam, lam0) <= 1e-10
    assert _rel(u, u0) <= 1e-10
    assert _rel(h, h0) <= 1e-10
    # recover from an explicit lambda (the oracle's) matches the oracle too
    u1, h1 = s.recover(ru, rh, lam0.reshape(lam.shape))
    assert _rel(u1, u0) <= 1e-12 and _rel(h1, h0) <= 1e-12
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 2)])
@pytest.mark.parametrize("reorth", [0, 1])
def test_iteration_count_matches_oracle(kind, p, reorth):
    """Same algorithm on both sides (FGMRES(30) + the same V-cycle; the
    oracle orthogonalises by modified Gram-Schmidt, the device by classical
    Gram-Schmidt once or twice, equal in exact arithmetic): the iteration
    counts to rtol 1e-8 agree within one."""
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-8, reorth=reorth)
    _, info = s.solve(ru, rh)
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S, coarse="gmg")
    _, info0 = gmres(lambda v: S @ v, prob.condensed_rhs(ru, rh), pc, restart=30, rtol=1e-8)
    assert abs(info["iters"] - info0["iters"]) <= 1
    s.close()


def test_device_entry_points_match_host_ones():
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = _solver(mesh, 2, tau, g, H, f, rtol=1e-12)
    lam, _ = s.solve(ru, rh)
    u, h = s.recover()
    lam_d = torch.empty((prob.n_facets, 3), dtype=torch.float64, device="cuda")
    s.solve_dev(_dev(ru), _dev(rh), lam_d)
    u_d = torch.empty((prob.N, 2, prob.np), dtype=torch.float64, device="cuda")
    h_d = torch.empty((prob.N, prob.np), dtype=torch.float64, device="cuda")
    s.recover_dev(_dev(ru), _dev(rh), lam_d, u_d, h_d)
    torch.cuda.synchronize()
    assert np.array_equal(lam_d.cpu().numpy(), lam)
    assert np.array_equal(u_d.cpu().numpy(), u) and np.array_equal(h_d.cpu().numpy(), h)
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 3), ("flat", 4), ("flat", 1)])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("reorth", [0, 1])
def test_mixed_precision(kind, p, mode, reorth):
    """FP32 inner FGMRES + FP32 V-cycle (mode 1) or with a BF16 operator copy in
    the smoother and V-cycle residual (mode 2), with FP64 iterative refinement,
    reaches the FP64 residual target; stated tolerance vs the oracle: 1e-8
    relative at rtol 1e-10 (the trace operator's condition number here is < 100)."""
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-10, precision=mode, reorth=reorth)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-10
    assert info["outer"] >= 2                  # refinement did happen
    assert _rel(lam, lam0) <= 1e-8 and _rel(u, u0) <= 1e-8 and _rel(h, h0) <= 1e-8
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 3), ("flat", 4), ("sphere", 3)])
def test_two_float_steps_match_fp64(kind, p):
    """Mixed modes do the FP64 steps (recovery, condensed right-hand side,
    refinement residual) in two-float arithmetic (about 48 significant bits):
    recovery from the same lambda agrees with the FP64 kernel to 1e-12, and a
    mixed solve to rtol 1e-11 meets it when its residual is measured with the
    FP64 operator.  The flat case (200 cells, 300 facets) leaves a ragged last
    block in both the 32-cell and the 256-facet kernels."""
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(10, n_coarsest=5)       # 200 cells, 300 facets
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
        tau = 8 * mesh.h / np.sqrt(g * H)
        n_p = (p + 1) * (p + 2) // 2
        rng = np.random.default_rng(1)
        ru = rng.standard_normal((mesh.n_cells, 2, n_p))
        rh = rng.standard_normal((mesh.n_cells, n_p))
        assert mesh.n_cells % 32 != 0
    else:
        mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s64 = _solver(mesh, p, tau, g, H, f, rtol=1e-12)
    s32 = _solver(mesh, p, tau, g, H, f, rtol=1e-11, precision=1)
    lam, _ = s64.solve(ru, rh)
    u64, h64 = s64.recover(ru, rh, lam)
    u32, h32 = s32.recover(ru, rh, lam)
    assert _rel(u32, u64) <= 1e-12 and _rel(h32, h64) <= 1e-12
    lam2, info = s32.solve(ru, rh)
    assert info["true_rel_res"] <= 1e-11
    gd = torch.empty(lam2.shape, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(gd)
    s64.condensed_rhs_dev(_dev(ru), _dev(rh), gd)
    s64.trace_apply_dev(_dev(lam2), yd)
    torch.cuda.synchronize()
    gh, yh = gd.cpu().numpy(), yd.cpu().numpy()
    assert np.linalg.norm(gh - yh) / np.linalg.norm(gh) <= 1.5e-11
    s64.close()
    s32.close()


@pytest.mark.parametrize("kind,p", [("flat", 3), ("sphere", 2)])
def test_page_locked_host_buffers_match_staged_path(kind, p):
    """Mixed handles read page-locked right-hand sides and write page-locked
    lambda / u / h in place (no staged copies); pageable numpy buffers take
    the staged path.  Same kernels and arithmetic: the results are identical,
    and hdg_recover(NULL, ...) afterwards still uses the solve's inputs."""
    import ctypes
    from paper_2004_09389_gb300 import _lib
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-10, precision=1)
    lam0, _ = s.solve(ru, rh)
    u0, h0 = s.recover()
    ru_p = torch.from_numpy(ru.copy()).pin_memory()
    rh_p = torch.from_numpy(rh.copy()).pin_memory()
    lam_p = torch.empty(lam0.shape, dtype=torch.float64).pin_memory()
    u_p = torch.empty(u0.shape, dtype=torch.float64).pin_memory()
    h_p = torch.empty(h0.shape, dtype=torch.float64).pin_memory()
    info = _lib.hdg_solve_info()
    _lib.check(s.h, s.lib.hdg_solve(s.h, ru_p.data_ptr(), rh_p.data_ptr(), lam_p.data_ptr(), ctypes.byref(info)))
    ru_p.zero_()                     # the recovery below must not read the caller's buffers
    rh_p.zero_()
    _lib.check(s.h, s.lib.hdg_recover(s.h, None, None, None, u_p.data_ptr(), h_p.data_ptr()))
    assert np.array_equal(lam_p.numpy(), lam0)
    assert np.array_equal(u_p.numpy(), u0) and np.array_equal(h_p.numpy(), h0)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_explicit_recover_inputs_leave_the_last_solve_selected(precision):
    """hdg_recover with explicit r_u, r_h (pageable, and page-locked on a
    mixed handle) serves that call only: a following hdg_recover with NULLs
    still uses the last solve's right-hand side.  One of r_u / r_h NULL is
    rejected."""
    import ctypes
    from paper_2004_09389_gb300 import _lib, HDGError
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = _solver(mesh, 2, tau, g, H, f, rtol=1e-10, precision=precision)
    lam, _ = s.solve(ru, rh)
    u0, h0 = s.recover()
    rng = np.random.default_rng(7)
    ru2, rh2 = rng.standard_normal(ru.shape), rng.standard_normal(rh.shape)
    u2_ref, h2_ref = prob.recover(lam.reshape(-1), ru2, rh2)
    u2, h2 = s.recover(ru2, rh2, lam)
    assert _rel(u2, u2_ref) <= 1e-12 and _rel(h2, h2_ref) <= 1e-12
    u1, h1 = s.recover()
    assert np.array_equal(u1, u0) and np.array_equal(h1, h0)
    ru_p = torch.from_numpy(ru2.copy()).pin_memory()
    rh_p = torch.from_numpy(rh2.copy()).pin_memory()
    u_p = torch.empty(u0.shape, dtype=torch.float64).pin_memory()
    h_p = torch.empty(h0.shape, dtype=torch.float64).pin_memory()
    _lib.check(s.h, s.lib.hdg_recover(s.h, ru_p.data_ptr(), rh_p.data_ptr(), None, u_p.data_ptr(), h_p.data_ptr()))
    assert np.array_equal(u_p.numpy(), u2) and np.array_equal(h_p.numpy(), h2)
    u1, h1 = s.recover()
    assert np.array_equal(u1, u0) and np.array_equal(h1, h0)
    with pytest.raises(HDGError) as ei:
        s.recover(ru2, None)
    assert ei.value.code == -1
    s.close()


@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 3), ("flat", 4), ("flat", 1)])
def test_fp64_fgmres_with_fp32_preconditioner(kind, p):
    """HDG_MIXED_FGMRES64: FP64 FGMRES (basis, orthogonalisation, residual,
    update, right-hand side and recovery in FP64) preconditioned by the FP32
    two-level V-cycle with an FP64 coarsest solve.  It reaches the FP64 residual
    target; stated tolerance vs the oracle: 1e-8 relative at rtol 1e-10; the
    FP32 preconditioner costs at most one iteration against the FP64 one."""
    from paper_2004_09389_gb300 import HDG_MIXED_FGMRES64
    mesh, prob, (tau, g, H, f), ru, rh = _case(kind, p)
    s = _solver(mesh, p, tau, g, H, f, rtol=1e-10, precision=HDG_MIXED_FGMRES64)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["true_rel_res"] <= 1e-10
    assert _rel(lam, lam0) <= 1e-8 and _rel(u, u0) <= 1e-8 and _rel(h, h0) <= 1e-8
    s64 = _solver(mesh, p, tau, g, H, f, rtol=1e-10)
    _, info64 = s64.solve(ru, rh)
    assert abs(info["iters"] - info64["iters"]) <= 1
    # the residual measured with the FP64 operator of the FP64 handle
    gd = torch.empty(lam.shape, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(gd)
    s64.condensed_rhs_dev(_dev(ru), _dev(rh), gd)
    s64.trace_apply_dev(_dev(lam), yd)
    torch.cuda.synchronize()
    gh, yh = gd.cpu().numpy(), yd.cpu().numpy()
    assert np.linalg.norm(gh - yh) / np.linalg.norm(gh) <= 1.5e-10
    s.close()
    s64.close()


def test_zero_rhs_and_nan_rhs():
    from paper_2004_09389_gb300 import HDGError
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 1)
    s = _solver(mesh, 1, tau, g, H, f)
    lam, info = s.solve(np.zeros_like(ru), np.zeros_like(rh))
    assert np.all(lam == 0) and info["iters"] == 0
    rh2 = rh.copy()
    rh2[3, 1] = np.nan
    with pytest.raises(HDGError) as ei:
        s.solve(ru, rh2)
    assert ei.value.code == -5          # HDG_ENAN
    # the handle stays usable afterwards
    lam, info = s.solve(ru, rh)
    assert info["true_rel_res"] <= 1e-8
    s.close()


def test_iteration_cap_reports_noconv():
    from paper_2004_09389_gb300 import HDGError
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = _solver(mesh, 2, tau, g, H, f, rtol=1e-14, max_iter=3)
    with pytest.raises(HDGError) as ei:
        s.solve(ru, rh)
    assert ei.value.code == -3          # HDG_ENOCONV
    lam, info = s.solve(ru, rh, allow_fail=True)
    assert info["iters"] == 3 and info["true_rel_res"] < 1.0
    s.close()


def test_invalid_arguments():
    from paper_2004_09389_gb300 import HDGError
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 1)
    for kw in ({"p": 5}, {"tau": -1.0}, {"restart": 0}, {"reorth": 2}):
        args = dict(p=1, tau=tau)
        args.update(kw)
        with pytest.raises(HDGError) as ei:
            _solver(mesh, args.pop("p"), args.pop("tau"), g, H, f, **args)
        assert ei.value.code == -1
    # open mesh: drop one cell
    bad = I.periodic_square(4)
    bad.cell_vertices = bad.cell_vertices[1:]
    bad.cell_shift = bad.cell_shift[1:]
    with pytest.raises(HDGError) as ei:
        _solver(bad, 1, 0.1, 1.0, 1.0, None)
    assert ei.value.code == -1
    # solve before condense
    s = _solver(mesh, 1, tau, g, H, f, condense=False)
    with pytest.raises(HDGError) as ei:
        s.solve(ru, rh)
    assert ei.value.code == -9
    s.close()


@pytest.mark.parametrize("kind", ["flat", "sphere"])
@pytest.mark.parametrize("p1_nu", [(2, 2), (3, 3), (1, 1)])
def test_precond_multi_block_p1_levels_match_oracle(kind, p1_nu, monkeypatch):
    """The P1 levels above the single-CTA tail: with the tail limited to 16
    vertices every other level runs in multi-block kernels, the patch-fused
    ones (sweep + residual + restriction going down, prolongation + two
    sweeps going up, ragged patches on three levels) where a level takes two
    or more sweeps.  FP64 matches the oracle; FP64 and FP32 match the unfused
    kernels up to summation order."""
    if kind == "flat":
        mesh = I.periodic_square_hierarchy(24, n_coarsest=3)       # P1 levels 576, 144, 36, 9
        g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    else:
        mesh = I.sphere_hierarchy(3, 1.0, r_coarsest=0)            # P1 levels 642, 162, 42, 12
        g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
    p = 1
    tau = 8 * mesh.h / np.sqrt(g * H)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    v = np.random.default_rng(5).standard_normal(prob.n_trace)
    monkeypatch.setenv("HDG_TAIL_MAX_VERTICES", "16")
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("HDG_P1_FUSED", fused)
        s = _solver(mesh, p, tau, g, H, f, precision=1, p1_nu_pre=p1_nu[0], p1_nu_post=p1_nu[1])
        z = torch.empty(prob.n_trace, dtype=torch.float64, device="cuda")
        z32 = torch.empty(prob.n_trace, dtype=torch.float32, device="cuda")
        s.precond_apply_dev(_dev(v), z)
        s.precond_apply32_dev(_dev(v.astype(np.float32)), z32)
        torch.cuda.synchronize()
        out[fused] = (z.cpu().numpy(), z32.cpu().numpy().astype(np.float64))
        s.close()
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator(), coarse="gmg", p1_nu=p1_nu)
    z0 = pc(v)
    assert _rel(out["1"][0], z0) <= 1e-12
    assert _rel(out["1"][0], out["0"][0]) <= 1e-14
    assert _rel(out["1"][1], out["0"][1]) <= 1e-6
    assert _rel(out["1"][1], z0) <= 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_set_tau_recondenses_in_place(precision, monkeypatch):
    """hdg_set_tau re-condenses the handle: operators, P1 levels and the
    single-CTA cycle's shared-memory image are rebuilt in place under the
    step graphs captured by the first solve.  The next solve equals that of a
    fresh handle built with the new tau (same kernels, same data: bit for bit)
    and the oracle's solution.  The coarse cycle is limited to 16 vertices so
    that the patch-fused P1 kernels run too."""
    monkeypatch.setenv("HDG_TAIL_MAX_VERTICES", "16")
    mesh = I.periodic_square_hierarchy(24, n_coarsest=3)
    g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
    p = 2
    tau1 = 8 * mesh.h / np.sqrt(g * H)
    tau2 = 2.5 * tau1
    prob2 = HDGProblem(mesh, p, tau=tau2, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(11)
    ru = rng.standard_normal((mesh.n_cells, 2, prob2.np))
    rh = rng.standard_normal((mesh.n_cells, prob2.np))
    s = _solver(mesh, p, tau1, g, H, f, precision=precision, rtol=1e-10)
    s.solve(ru, rh)
    s.set_tau(tau2)
    lam, info = s.solve(ru, rh)
    u, h = s.recover()
    fresh = _solver(mesh, p, tau2, g, H, f, precision=precision, rtol=1e-10)
    lam_f, info_f = fresh.solve(ru, rh)
    u_f, h_f = fresh.recover()
    assert info["iters"] == info_f["iters"]
    assert np.array_equal(lam, lam_f) and np.array_equal(u, u_f) and np.array_equal(h, h_f)
    (u0, h0), lam0 = prob2.solve_condensed(ru, rh)
    tol = 1e-8 if precision else 1e-9
    assert _rel(lam, lam0.reshape(lam.shape)) <= tol and _rel(u, u0) <= tol and _rel(h, h0) <= tol
    s.close()
    fresh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_kernel_accounting_keeps_the_result(precision):
    """With timing on, every launch is bracketed by CUDA events and the
    Arnoldi steps run as direct launches instead of replayed graphs: the
    solution is bit-identical, the per-category launch counts equal those the
    graphs report, and every category the solve uses gets time."""
    mesh, prob, (tau, g, H, f), ru, rh = _case("flat", 2)
    s = _solver(mesh, 2, tau, g, H, f, precision=precision, rtol=1e-10)
    s.solve(ru, rh)                       # step graphs captured
    s.profile_enable(False)               # counters reset, timing off
    lam_g, info_g = s.solve(ru, rh)
    counts_g = {k: v[1] for k, v in s.profile_read().items()}
    s.profile_enable(True)
    lam_t, info_t = s.solve(ru, rh)
    prof = s.profile_read()
    s.close()
    assert info_g["iters"] == info_t["iters"] and np.array_equal(lam_g, lam_t)
    assert {k: v[1] for k, v in prof.items()} == counts_g
    for k in ("apply64" if precision == 0 else "apply32", "p1", "krylov", "rhs", "layout"):
        assert prof[k][1] > 0 and prof[k][0] > 0.0, (k, prof[k])
