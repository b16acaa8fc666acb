"""Learned facet-patch smoother on the GPU (an extension beyond the paper).

* loss and gradient of the library's own forward / backward kernels agree with
  the oracle's (FP64, hand-written backward pinned by finite differences) to
  FP32 accuracy (relative 2e-3 on the gradient, 1e-4 on the loss);
* zero weights reproduce the plain solver (the learned sweep is then the
  damped block-Jacobi sweep);
* garbage weights trigger the stall fallback and the solve still converges;
* after training on residuals from plain solves, held-out solves need fewer
  FGMRES iterations than without the network when the inner solve is long
  (inner_rtol 1e-7: one FP32 inner solve does most of the work); the gain is
  printed.  With the default short inner solves (1e-4, ~5 iterations each) the
  learned sweep does not remove an iteration: it tightens the contraction of
  the last sweep, which shows only over longer runs.
"""
import math

import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem
from oracle import learned as LN
from oracle.solver import TwoLevelPreconditioner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build
    build.build()


def _flat(n, p):
    mesh = I.periodic_square_hierarchy(n, side=5.12e6 * n / 256, n_coarsest=4)
    g, H, f0 = 9.81, 1e3, 1e-4
    tau = 8 * mesh.h / math.sqrt(g * H)
    return mesh, tau, g, H, I.coriolis_flat(mesh, f0)


@pytest.mark.parametrize("p,hid", [(1, 32), (2, 64)])
def test_gradient_matches_oracle(p, hid):
    from paper_2004_09389_gb300 import HDGSolver
    mesh, tau, g, H, f = _flat(8, p)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=1)
    npar = s.learned_init(hidden=hid, capacity=4)
    rng = np.random.default_rng(0)
    theta = (0.3 * rng.standard_normal(npar)).astype(np.float32)
    s.set_learned_params(theta)
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)
    S = prob.trace_operator().tocsr()
    pc = TwoLevelPreconditioner(prob, mesh, S)
    pp = p + 1
    Dinv = np.stack([pc.Dinv[e * pp:(e + 1) * pp][:, e * pp:(e + 1) * pp].toarray() for e in range(prob.n_facets)])
    nbr = LN.library_neighbours(prob)
    R = rng.standard_normal((2, prob.n_trace)).astype(np.float32)
    L0, g0 = LN.loss_and_grad(theta.astype(np.float64), R.astype(np.float64), S, nbr, Dinv, hid, pp, 2.0 / 3.0)
    L1, g1 = s.learned_loss_grad_dev(torch.from_numpy(R.reshape(2, prob.n_facets, pp)).cuda())
    assert abs(L1 - L0) <= 1e-4 * abs(L0)
    assert np.linalg.norm(g1 - g0) <= 2e-3 * np.linalg.norm(g0)
    s.close()


def _rhs(mesh, p, seed):
    ru, rh = I.gaussian_field_rhs(mesh, p, seed, grid=128, kmax=mesh.n_vertices ** 0.5 / 2)
    return torch.from_numpy(ru).cuda(), torch.from_numpy(rh).cuda()


def test_zero_weights_reproduce_the_plain_solver():
    from paper_2004_09389_gb300 import HDGSolver
    mesh, tau, g, H, f = _flat(32, 2)
    s = HDGSolver(mesh, 2, tau, g, H, f_vertex=f, precision=1, rtol=1e-8)
    s.learned_init(hidden=32, capacity=4)
    s.set_learned_params(np.zeros(s.n_learned_params, np.float32))
    ru, rh = _rhs(mesh, 2, 3)
    lam0 = torch.zeros((s.n_facets, 3), dtype=torch.float64, device="cuda")
    lam1 = torch.zeros_like(lam0)
    i0 = s.solve_dev(ru, rh, lam0)
    s.learned_enable(True)
    i1 = s.solve_dev(ru, rh, lam1)
    torch.cuda.synchronize()
    assert i1["iters"] == i0["iters"] and i1["fallback_used"] == 0
    assert (lam1 - lam0).norm().item() <= 1e-6 * lam0.norm().item()
    s.close()


def test_bad_weights_fall_back_and_converge():
    from paper_2004_09389_gb300 import HDGSolver
    mesh, tau, g, H, f = _flat(32, 2)
    s = HDGSolver(mesh, 2, tau, g, H, f_vertex=f, precision=1, rtol=1e-8)
    s.learned_init(hidden=32, capacity=4)
    s.set_learned_params((50.0 * np.random.default_rng(1).standard_normal(s.n_learned_params)).astype(np.float32))
    s.learned_enable(True)
    ru, rh = _rhs(mesh, 2, 4)
    lam = torch.zeros((s.n_facets, 3), dtype=torch.float64, device="cuda")
    info = s.solve_dev(ru, rh, lam)
    assert info["fallback_used"] == 1 and info["true_rel_res"] <= 1e-8
    s.close()


def test_training_improves_the_preconditioner():
    """Trained on residuals of plain solves, the learned sweep lowers the
    contraction ||v - S V(v)|| / ||v|| of one preconditioner application on
    held-out right-hand sides; iteration counts do not get worse."""
    from paper_2004_09389_gb300 import HDGSolver
    mesh, tau, g, H, f = _flat(32, 2)
    s = HDGSolver(mesh, 2, tau, g, H, f_vertex=f, precision=1, rtol=1e-8)
    s64 = HDGSolver(mesh, 2, tau, g, H, f_vertex=f)
    s.learned_init(hidden=32, capacity=512, seed=7)
    for k in range(8):
        n = s.learned_collect_dev(*_rhs(mesh, 2, 100 + k))
    assert n >= 64
    l0, l1 = s.learned_train(steps=600, batch=8, lr=2e-3)
    assert l1 < 0.8 * l0

    def contraction(on):
        s.learned_enable(on)
        acc = []
        for k in range(4):
            ru, rh = _rhs(mesh, 2, 900 + k)
            gv = torch.empty((s.n_facets, 3), dtype=torch.float64, device="cuda")
            s64.condensed_rhs_dev(ru, rh, gv)
            v32 = gv.float().contiguous()
            z32 = torch.empty_like(v32)
            s.precond_apply32_dev(v32, z32)
            Sz = torch.empty_like(gv)
            s64.trace_apply_dev(z32.double().contiguous(), Sz)
            torch.cuda.synchronize()
            acc.append(((gv - Sz).norm() / gv.norm()).item())
        return float(np.mean(acc))

    c_plain, c_learned = contraction(False), contraction(True)
    plain, learned = 0, 0
    for k in range(4):
        ru, rh = _rhs(mesh, 2, 900 + k)
        lam = torch.zeros((s.n_facets, 3), dtype=torch.float64, device="cuda")
        s.learned_enable(False)
        a = s.solve_dev(ru, rh, lam)
        s.learned_enable(True)
        b = s.solve_dev(ru, rh, lam)
        assert b["true_rel_res"] <= 1e-8
        plain += a["iters"]
        learned += b["iters"]
    print(f"\nlearned smoother: training loss {l0:.3f} -> {l1:.3f}; contraction of one preconditioner "
          f"application {c_plain:.3f} -> {c_learned:.3f}; inner iterations on 4 held-out solves {plain} -> {learned}")
    assert c_learned < 0.95 * c_plain
    assert learned <= plain
    s.close()
    s64.close()


@pytest.mark.parametrize("p,hid,n", [(1, 32, 8), (3, 64, 8), (2, 64, 32), (4, 32, 32)])
def test_tensor_core_network_matches_fp32(p, hid, n):
    """The network's three layers as tcgen05 GEMMs over tiles of 128 facets
    (BF16 weights and activations, FP32 accumulation in tensor memory) against
    the FP32 network on the CUDA cores, one preconditioner application with the
    learned sweep: the difference is at most 3 % of the learned part (the FP32
    output minus the output with the network's output layer zeroed; BF16 keeps
    8 significant bits per rounding, three layers deep); the learned sweep is
    the last post-smoothing sweep, so that part is a small share of the output.  n = 8 leaves a ragged
    last tile (192 facets), n = 32 fills 24 tiles.  A full solve with the
    tensor-core sweep still reaches its tolerance."""
    from paper_2004_09389_gb300 import HDGSolver
    mesh, tau, g, H, f = _flat(n, p)
    s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, precision=1, rtol=1e-8)
    npar = s.learned_init(hidden=hid, capacity=4)
    rng = np.random.default_rng(1)
    theta = (0.3 * rng.standard_normal(npar)).astype(np.float32)
    s.set_learned_params(theta)
    pp = p + 1
    nt = s.n_facets * pp
    v = torch.from_numpy(np.random.default_rng(2).standard_normal(nt).astype(np.float32)).cuda()

    def z_of(tc):
        s.learned_enable(True, tensor_cores=tc)
        z = torch.empty_like(v)
        s.precond_apply32_dev(v, z)
        torch.cuda.synchronize()
        return z.cpu().numpy().astype(np.float64)

    z32 = z_of(False)
    ztc = z_of(True)
    shapes = LN.param_shapes(5 * pp, hid, pp)
    n_out = int(np.prod(shapes[-2][1])) + int(np.prod(shapes[-1][1]))
    theta0 = theta.copy()
    theta0[-n_out:] = 0.0                       # W3 and b3: the learned part off
    s.set_learned_params(theta0)
    zlin = z_of(False)
    part = np.linalg.norm(z32 - zlin)
    # the learned sweep is the last post-smoothing sweep: its share of the
    # preconditioner's output is small but well above rounding
    assert part > 1e-3 * np.linalg.norm(z32)
    assert np.all(np.isfinite(ztc))
    ratio = np.linalg.norm(ztc - z32) / part
    print(f"p={p} hidden={hid} n={n}: |z_tc - z_fp32| / |learned part| = {ratio:.2e}")
    assert ratio <= 0.03
    # a full solve with the tensor-core sweep (the stall fallback may take over)
    s.set_learned_params(theta)
    s.learned_enable(True, tensor_cores=True)
    ru = np.random.default_rng(3).standard_normal((mesh.n_cells, 2, (p + 1) * (p + 2) // 2))
    rh = np.random.default_rng(4).standard_normal((mesh.n_cells, (p + 1) * (p + 2) // 2))
    _, info = s.solve(ru, rh)
    assert info["true_rel_res"] <= 1e-8
    s.close()
