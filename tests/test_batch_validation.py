"""Argument checks of the merged-batch entry points on the CPU: each runs on
the host before the first CUDA call, so malformed calls are refused with
HDG_EINVAL and a message, without a GPU; NULL batches are handled."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2004_09389_gb300 import _lib
    return _lib.load()


def _err(lib):
    return (lib.hdg_last_error(None) or b"").decode()


def test_create_refuses_bad_arguments(lib):
    from paper_2004_09389_gb300 import _lib
    out = ctypes.c_void_p(1234)
    assert lib.hdg_batch_create(None, 1, None) == _lib.HDG_EINVAL
    assert "out is NULL" in _err(lib)
    assert lib.hdg_batch_create(None, 1, ctypes.byref(out)) == _lib.HDG_EINVAL
    assert out.value is None                        # cleared before the checks
    assert "at least one handle" in _err(lib)
    hs = (ctypes.c_void_p * 1)()
    assert lib.hdg_batch_create(hs, 0, ctypes.byref(out)) == _lib.HDG_EINVAL


def test_solve_stats_destroy_refuse_null(lib):
    from paper_2004_09389_gb300 import _lib
    info = (_lib.hdg_solve_info * 1)()
    assert lib.hdg_batch_solve_dev(None, None, None, None, info) == _lib.HDG_EINVAL
    assert "batch is NULL" in _err(lib)
    assert lib.hdg_batch_solve(None, None, None, None, info) == _lib.HDG_EINVAL
    stats = (ctypes.c_int64 * 8)()
    assert lib.hdg_batch_stats(None, stats) == _lib.HDG_EINVAL
    assert lib.hdg_batch_destroy(None) == _lib.HDG_OK
