"""ctypes binding of ``include/hdg.h`` (argument marshalling only).

Every numerical step runs in the CUDA library ``lib/libhdg.so``; if it is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhdg.so")

HDG_OK, HDG_EINVAL, HDG_ESINGULAR, HDG_ENOCONV = 0, -1, -2, -3
HDG_EBREAKDOWN, HDG_ENAN, HDG_ECUDA, HDG_ETIMEOUT, HDG_ENOMEM, HDG_ESTATE = -4, -5, -6, -7, -8, -9
HDG_FP64, HDG_MIXED_FP32, HDG_MIXED_BF16, HDG_MIXED_FGMRES64 = 0, 1, 2, 3
HDG_IMEX_THETA, HDG_IMEX_ARS2, HDG_IMEX_SSP2, HDG_IMEX_ARS3 = 0, 1, 2, 3
IMEX_SCHEMES = {"theta": HDG_IMEX_THETA, "ARS2": HDG_IMEX_ARS2, "SSP2": HDG_IMEX_SSP2, "ARS3": HDG_IMEX_ARS3}

ERROR_NAMES = {0: "HDG_OK", -1: "HDG_EINVAL", -2: "HDG_ESINGULAR", -3: "HDG_ENOCONV",
               -4: "HDG_EBREAKDOWN", -5: "HDG_ENAN", -6: "HDG_ECUDA", -7: "HDG_ETIMEOUT",
               -8: "HDG_ENOMEM", -9: "HDG_ESTATE"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class hdg_mesh_level(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_cells", C.c_int32), ("dim", C.c_int32),
                ("vertex_xyz", _dp), ("cell_vertices", _ip), ("cell_shift", _dp), ("parent", _ip)]


class hdg_mesh_desc(C.Structure):
    _fields_ = [("fine", hdg_mesh_level), ("n_coarse", C.c_int32), ("coarse", C.POINTER(hdg_mesh_level))]


class hdg_params(C.Structure):
    _fields_ = [("p", C.c_int32), ("tau", C.c_double), ("g", C.c_double), ("H", C.c_double),
                ("tau_s", C.c_double), ("f_vertex", _dp), ("precision", C.c_int32), ("rtol", C.c_double),
                ("restart", C.c_int32), ("max_iter", C.c_int32), ("n_pre", C.c_int32), ("n_post", C.c_int32),
                ("omega", C.c_double), ("p1_nu_pre", C.c_int32), ("p1_nu_post", C.c_int32),
                ("p1_omega", C.c_double), ("inner_rtol", C.c_double), ("coarse_mode", C.c_int32),
                ("reorth", C.c_int32), ("smoother", C.c_int32), ("cheb_theta", C.c_double),
                ("cheb_delta2", C.c_double), ("cheb_steps", C.c_int32), ("flux", C.c_int32),
                ("n_coarse", C.c_int32), ("keep_rhs", C.c_int32)]


class hdg_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("status", C.c_int32), ("fallback_used", C.c_int32),
                ("true_rel_res", C.c_double), ("est_rel_res", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class HDGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None
EXPORTS = ["hdg_default_params", "hdg_setup", "hdg_condense", "hdg_set_tau", "hdg_solve", "hdg_solve_dev",
           "hdg_solve_recover",
           "hdg_recover", "hdg_recover_dev", "hdg_trace_apply_dev", "hdg_condensed_rhs_dev",
           "hdg_precond_apply_dev", "hdg_get_sizes", "hdg_get_facets", "hdg_get_cell_schur", "hdg_destroy",
           "hdg_last_error", "hdg_profile_enable", "hdg_profile_read", "hdg_condensed_rhs_noalloc_dev",
           "hdg_solve_batch_dev", "hdg_autotune", "hdg_get_stream", "hdg_learned_init",
           "hdg_learned_collect_dev", "hdg_learned_train", "hdg_learned_params", "hdg_learned_enable",
           "hdg_learned_loss_grad_dev", "hdg_precond_apply32_dev", "hdg_fma_rate",
           "hdg_imex_init", "hdg_imex_rates_dev", "hdg_imex_step_dev", "hdg_get_chebyshev",
           "hdg_get_rt0_chebyshev", "hdg_batch_create", "hdg_batch_solve_dev", "hdg_batch_solve", "hdg_batch_stats",
           "hdg_batch_destroy"]

HDG_PROF_N = 16
PROF_NAMES = ["apply64", "residual64", "smooth64", "smooth_first64", "apply32", "residual32", "smooth32",
              "smooth_first32", "transfer", "p1", "krylov", "rhs", "recover", "layout", "condense", "imex"]


def load() -> C.CDLL:
    """Load ``lib/libhdg.so`` (build it first with ``build.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2004_09389_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.hdg_default_params.argtypes = [C.POINTER(hdg_params)]
    lib.hdg_default_params.restype = None
    lib.hdg_setup.argtypes = [C.POINTER(hdg_mesh_desc), C.POINTER(hdg_params), vp, C.POINTER(vp)]
    for name in ("hdg_condense", "hdg_destroy"):
        getattr(lib, name).argtypes = [vp]
    lib.hdg_set_tau.argtypes = [vp, C.c_double]
    for name in ("hdg_solve", "hdg_solve_dev"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp, C.POINTER(hdg_solve_info)]
    lib.hdg_solve_recover.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(hdg_solve_info)]
    for name in ("hdg_recover", "hdg_recover_dev"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp]
    lib.hdg_trace_apply_dev.argtypes = [vp, vp, vp]
    lib.hdg_condensed_rhs_dev.argtypes = [vp, vp, vp, vp]
    lib.hdg_condensed_rhs_noalloc_dev.argtypes = [vp, vp, vp, vp]
    lib.hdg_precond_apply_dev.argtypes = [vp, vp, vp]
    lib.hdg_precond_apply32_dev.argtypes = [vp, vp, vp]
    lib.hdg_get_sizes.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.hdg_get_facets.argtypes = [vp, vp, vp, vp]
    lib.hdg_get_cell_schur.argtypes = [vp, vp]
    lib.hdg_solve_batch_dev.argtypes = [vp, C.c_int, vp, vp, vp, C.POINTER(hdg_solve_info), C.c_int]
    lib.hdg_batch_create.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.hdg_batch_solve_dev.argtypes = [vp, vp, vp, vp, C.POINTER(hdg_solve_info)]
    lib.hdg_batch_solve.argtypes = [vp, vp, vp, vp, C.POINTER(hdg_solve_info)]
    lib.hdg_batch_stats.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.hdg_batch_destroy.argtypes = [vp]
    lib.hdg_autotune.argtypes = [vp, vp]
    lib.hdg_get_stream.argtypes = [vp]
    lib.hdg_learned_init.argtypes = [vp, C.c_int, C.c_int, C.c_uint64, vp]
    lib.hdg_learned_collect_dev.argtypes = [vp, vp, vp, vp]
    lib.hdg_learned_train.argtypes = [vp, C.c_int, C.c_int, C.c_double, vp, vp]
    lib.hdg_learned_params.argtypes = [vp, vp, C.c_int]
    lib.hdg_learned_enable.argtypes = [vp, C.c_int]
    lib.hdg_learned_loss_grad_dev.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.hdg_get_stream.restype = vp
    lib.hdg_profile_enable.argtypes = [vp, C.c_int]
    lib.hdg_profile_read.argtypes = [vp, vp, vp]
    lib.hdg_fma_rate.argtypes = [C.c_int, vp]
    lib.hdg_get_chebyshev.argtypes = [vp, vp, vp, vp]
    lib.hdg_get_rt0_chebyshev.argtypes = [vp, vp, vp, vp]
    lib.hdg_imex_init.argtypes = [vp, vp]
    lib.hdg_imex_rates_dev.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.hdg_imex_step_dev.argtypes = [vp, C.c_int, C.c_double, C.c_double, vp, vp, C.POINTER(hdg_solve_info)]
    lib.hdg_last_error.argtypes = [vp]
    lib.hdg_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("hdg_default_params", "hdg_last_error", "hdg_get_stream"):
            getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor (None -> 0)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _level(mesh, keep: list, parent=None) -> hdg_mesh_level:
    xyz = np.ascontiguousarray(mesh.vertex_xyz, dtype=np.float64)
    cv = np.ascontiguousarray(mesh.cell_vertices, dtype=np.int32)
    sh = None if mesh.cell_shift is None else np.ascontiguousarray(mesh.cell_shift, dtype=np.float64)
    par = None if parent is None else np.ascontiguousarray(parent, dtype=np.int32)
    keep += [xyz, cv, sh, par]
    return hdg_mesh_level(int(xyz.shape[0]), int(cv.shape[0]), int(mesh.dim),
                          xyz.ctypes.data_as(_dp), cv.ctypes.data_as(_ip),
                          None if sh is None else sh.ctypes.data_as(_dp),
                          None if par is None else par.ctypes.data_as(_ip))


def make_mesh_desc(mesh, keep: list) -> hdg_mesh_desc:
    """Descriptor of a mesh object with ``dim, vertex_xyz, cell_vertices,
    cell_shift`` and a list ``levels`` of coarse levels carrying ``parent``."""
    levels = list(getattr(mesh, "levels", []) or [])
    arr = (hdg_mesh_level * max(len(levels), 1))()
    for i, lev in enumerate(levels):
        arr[i] = _level(lev, keep, lev.parent)
    keep.append(arr)
    return hdg_mesh_desc(_level(mesh, keep), len(levels), arr if levels else None)


def default_params() -> hdg_params:
    prm = hdg_params()
    load().hdg_default_params(C.byref(prm))
    return prm


def check(handle, rc: int, allow=()) -> int:
    if rc != 0 and rc not in allow:
        msg = load().hdg_last_error(handle)
        raise HDGError(rc, msg.decode() if msg else "")
    return rc


def fma_rate(nbytes: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU for FP64 (8) or FP32 (4)."""
    out = C.c_double(0.0)
    check(None, load().hdg_fma_rate(int(nbytes), C.byref(out)))
    return out.value
