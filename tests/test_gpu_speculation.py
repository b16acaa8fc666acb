"""Arnoldi steps queued ahead do not change results.

An FGMRES cycle may queue step j + 1 before step j's residual estimate reaches
the host (HDG_SPECULATE; read once per process).  A step queued ahead of a
converged one runs for nothing and nothing of it is used, so every solve must
return the same lambda, bit for bit, with the switch on (default) and off.  The
child processes run three solves in a row on each handle, so that readback
slots left pending by one solve's last cycle are met again by the next.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build
    build.build()


CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    import hdg_inputs as I
    from paper_2004_09389_gb300 import HDGSolver, HDG_FP64, HDG_MIXED_FP32
    out = sys.argv[1]
    res = {}
    for name, kind, p, prec in (("mixed_flat", "flat", 2, HDG_MIXED_FP32), ("fp64_flat", "flat", 3, HDG_FP64),
                                ("mixed_sphere", "sphere", 3, HDG_MIXED_FP32)):
        if kind == "flat":
            mesh = I.periodic_square_hierarchy(16, n_coarsest=4)
            g, H, f = 1.3, 0.7, I.coriolis_flat(mesh, 1.0)
        else:
            mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)
            g, H, f = 1.0, 1.0, I.coriolis_sphere(mesh, 0.5)
        tau = 8 * mesh.h / np.sqrt(g * H)
        s = HDGSolver(mesh, p, tau, g, H, f_vertex=f, rtol=1e-12, precision=prec, inner_rtol=1e-3)
        rng = np.random.default_rng(5)
        for k in range(3):
            ru = torch.from_numpy(rng.standard_normal((s.n_cells, 2, s.n_p))).cuda()
            rh = torch.from_numpy(rng.standard_normal((s.n_cells, s.n_p))).cuda()
            lam = torch.zeros((s.n_facets, p + 1), dtype=torch.float64, device="cuda")
            info = s.solve_dev(ru, rh, lam)
            torch.cuda.synchronize()
            res[f"{name}_{k}"] = lam.cpu().numpy()
            res[f"{name}_{k}_iters"] = np.array([info["iters"], info["outer"]])
        s.close()
    np.savez(out, **res)
""")


def _run(tmp_path, spec):
    out = str(tmp_path / f"lam_{spec}.npz")
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    if spec == "off":
        env["HDG_SPECULATE"] = "0"
    else:
        env.pop("HDG_SPECULATE", None)
    subprocess.run([sys.executable, "-c", CHILD, out], cwd=ROOT, env=env, check=True, timeout=600)
    return np.load(out)


def test_queued_ahead_steps_leave_results_unchanged(tmp_path):
    on = _run(tmp_path, "on")
    off = _run(tmp_path, "off")
    assert sorted(on.files) == sorted(off.files)
    for k in on.files:
        assert np.array_equal(on[k], off[k]), k
    # the inner solves ran several Arnoldi steps, so steps were queued ahead
    assert all(on[f"mixed_flat_{k}_iters"][0] >= 4 for k in range(3))
