"""hdg_condensed_rhs_noalloc_dev: step 1 with its scratch in a fixed device array.

Some callers cannot let the library allocate device memory once they are
running: applications that hand all device memory to their own pool at
start-up, or that cannot take the device-wide synchronisation that cudaMalloc
and cudaFree may cause on their other streams.  For them the condensed
right-hand side has a variant whose scratch is a static array in the library's
device image, placed on the device by hdg_setup.  This test calls it through
the C ABI, twice in a row with different right-hand sides (the array keeps the
previous call's contents), and checks each result against
hdg_condensed_rhs_dev to the 1e-12 relative tolerance of the other parity
tests; it checks that the device's free memory does not change across the
first call on a fresh handle, and the size limit.  It runs last (file name)
and works alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import hdg_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09389_gb300 import build, _lib
    build.build()
    return _lib


def test_noalloc_rhs_matches_existing_entry_point(lib):
    from paper_2004_09389_gb300 import HDGSolver
    mesh = I.sphere_hierarchy(3, 1.0, r_coarsest=1)          # 1280 cells: several tiles, ragged tail
    p = 3
    s = HDGSolver(mesh, p, 8 * mesh.h, 1.0, 1.0, f_vertex=I.coriolis_sphere(mesh, 0.5))
    rng = np.random.default_rng(11)
    free_before = None
    for call in range(2):
        ru = torch.from_numpy(rng.standard_normal((s.n_cells, 2, s.n_p))).cuda()
        rh = torch.from_numpy(rng.standard_normal((s.n_cells, s.n_p))).cuda()
        g_ref = torch.empty((s.n_facets, p + 1), dtype=torch.float64, device="cuda")
        g_new = torch.full((s.n_facets, p + 1), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()         # inputs were written on PyTorch's stream; the calls run on the handle's
        lib.check(s.h, s.lib.hdg_condensed_rhs_dev(s.h, ru.data_ptr(), rh.data_ptr(), g_ref.data_ptr()))
        torch.cuda.synchronize()
        if call == 0:
            free_before = torch.cuda.mem_get_info()[0]
        lib.check(s.h, s.lib.hdg_condensed_rhs_noalloc_dev(s.h, ru.data_ptr(), rh.data_ptr(), g_new.data_ptr()))
        torch.cuda.synchronize()
        if call == 0:
            # the first call on a fresh handle loads nothing and allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        a, b = g_new.cpu().numpy(), g_ref.cpu().numpy()
        assert np.isfinite(a).all(), f"call {call}: output not fully written"
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), f"call {call}"
    s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    from paper_2004_09389_gb300 import HDGSolver
    mesh = I.periodic_square_hierarchy(320, n_coarsest=5)      # 204,800 cells; p = 4 needs 4.6M doubles
    s = HDGSolver(mesh, 4, 0.01, 1.0, 1.0, condense=False)
    rc = s.lib.hdg_condensed_rhs_noalloc_dev(s.h, ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1))
    assert rc == lib.HDG_EINVAL
    assert b"exceeds" in s.lib.hdg_last_error(s.h) or b"more than the fixed" in s.lib.hdg_last_error(s.h)
    s.close()
