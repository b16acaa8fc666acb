"""One HDG solver handle (argument marshalling around ``include/hdg.h``)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _torch():
    try:
        import torch
        if torch.cuda.is_available():
            return torch
    except ImportError:
        pass
    return None


class HDGSolver:
    """Handle for one mesh and one parameter set.

    ``mesh`` is any object with ``dim``, ``vertex_xyz``, ``cell_vertices``,
    ``cell_shift`` and an optional list ``levels`` of coarse P1 levels (each with
    ``parent``).  Keyword arguments override the fields of ``hdg_params``.
    ``stream``: a ``torch.cuda.Stream`` (or a raw ``cudaStream_t`` value) for the
    handle's work; by default the handle creates its own stream (PyTorch hands
    out streams from a small pool, so many handles would share them).
    ``*_dev`` calls are ordered after the work already queued on PyTorch's
    current stream, and that stream waits for them, so tensors can be used
    right before and after the call.
    """

    def __init__(self, mesh, p: int, tau: float, g: float = 1.0, H: float = 1.0, f_vertex=None,
                 stream=None, condense: bool = True, **params):
        self.lib = L.load()
        prm = L.default_params()
        prm.p, prm.tau, prm.g, prm.H = int(p), float(tau), float(g), float(H)
        self._keep = []
        if f_vertex is not None:
            fv = np.ascontiguousarray(f_vertex, dtype=np.float64)
            self._keep.append(fv)
            prm.f_vertex = fv.ctypes.data_as(C.POINTER(C.c_double))
        for k, v in params.items():
            if not hasattr(prm, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(prm, k, v)
        desc = L.make_mesh_desc(mesh, self._keep)
        h = C.c_void_p()
        torch = _torch()
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        rc = self.lib.hdg_setup(C.byref(desc), C.byref(prm), C.c_void_p(raw), C.byref(h))
        self._keep = []
        if rc != 0:
            raise L.HDGError(rc, self.lib.hdg_last_error(None).decode())
        self.h = h
        self.p = int(p)
        if stream is None and torch is not None:
            stream = torch.cuda.ExternalStream(self.lib.hdg_get_stream(h))
        self.stream = stream
        sz = (C.c_int64 * 6)()
        L.check(h, self.lib.hdg_get_sizes(h, sz))
        self.n_cells, self.n_facets, self.n_trace, self.n_p, self.m, self.n_levels = (int(v) for v in sz)
        if condense:
            self.condense()

    # ---------------------------------------------------------------- lifecycle
    def condense(self) -> None:
        L.check(self.h, self.lib.hdg_condense(self.h))

    def set_tau(self, tau: float) -> None:
        L.check(self.h, self.lib.hdg_set_tau(self.h, C.c_double(tau)))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.hdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- host buffers
    def solve(self, r_u: np.ndarray, r_h: np.ndarray, allow_fail: bool = False):
        """Steps 1-2 from host arrays; returns (lambda [n_facets, p+1], info dict)."""
        ru = np.ascontiguousarray(r_u, dtype=np.float64)
        rh = np.ascontiguousarray(r_h, dtype=np.float64)
        assert ru.shape == (self.n_cells, 2, self.n_p) and rh.shape == (self.n_cells, self.n_p)
        lam = np.empty((self.n_facets, self.n_trace // self.n_facets))   # p+1 (upwind) or 2(p+1) (Lax-Friedrichs)
        info = L.hdg_solve_info()
        rc = self.lib.hdg_solve(self.h, ru.ctypes.data, rh.ctypes.data, lam.ctypes.data, C.byref(info))
        L.check(self.h, rc, allow=(L.HDG_ENOCONV, L.HDG_EBREAKDOWN) if allow_fail else ())
        return lam, info.as_dict()

    def solve_recover(self, r_u: np.ndarray, r_h: np.ndarray, allow_fail: bool = False):
        """Steps 1-3 from host arrays in one call (hdg_solve_recover); returns
        (lambda, u, h, info dict)."""
        ru = np.ascontiguousarray(r_u, dtype=np.float64)
        rh = np.ascontiguousarray(r_h, dtype=np.float64)
        assert ru.shape == (self.n_cells, 2, self.n_p) and rh.shape == (self.n_cells, self.n_p)
        lam = np.empty((self.n_facets, self.n_trace // self.n_facets))
        u = np.empty((self.n_cells, 2, self.n_p))
        h = np.empty((self.n_cells, self.n_p))
        info = L.hdg_solve_info()
        rc = self.lib.hdg_solve_recover(self.h, ru.ctypes.data, rh.ctypes.data, lam.ctypes.data, u.ctypes.data,
                                        h.ctypes.data, C.byref(info))
        L.check(self.h, rc, allow=(L.HDG_ENOCONV, L.HDG_EBREAKDOWN) if allow_fail else ())
        return lam, u, h, info.as_dict()

    def recover(self, r_u=None, r_h=None, lam=None):
        """Step 3 from host arrays; None selects the last solve's data."""
        u = np.empty((self.n_cells, 2, self.n_p))
        h = np.empty((self.n_cells, self.n_p))
        ru = None if r_u is None else np.ascontiguousarray(r_u, dtype=np.float64)
        rh = None if r_h is None else np.ascontiguousarray(r_h, dtype=np.float64)
        lm = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
        rc = self.lib.hdg_recover(self.h, L._ptr(ru), L._ptr(rh), L._ptr(lm), u.ctypes.data, h.ctypes.data)
        L.check(self.h, rc)
        return u, h

    # ---------------------------------------------------------------- device buffers
    def _ordered(self, fn, *args):
        """Run a *_dev call on the handle's stream, ordered with PyTorch's current stream."""
        torch = _torch()
        own = hasattr(self.stream, "wait_stream") and torch is not None
        if own:
            cur = torch.cuda.current_stream()
            self.stream.wait_stream(cur)
        rc = fn(self.h, *args)
        if own:
            cur.wait_stream(self.stream)
        return rc

    def solve_dev(self, r_u, r_h, lam, allow_fail: bool = False) -> dict:
        info = L.hdg_solve_info()
        rc = self._ordered(self.lib.hdg_solve_dev, L._ptr(r_u), L._ptr(r_h), L._ptr(lam), C.byref(info))
        L.check(self.h, rc, allow=(L.HDG_ENOCONV, L.HDG_EBREAKDOWN) if allow_fail else ())
        return info.as_dict()

    def recover_dev(self, r_u, r_h, lam, u, h) -> None:
        L.check(self.h, self._ordered(self.lib.hdg_recover_dev, L._ptr(r_u), L._ptr(r_h), L._ptr(lam), L._ptr(u),
                                      L._ptr(h)))

    def trace_apply_dev(self, x, y) -> None:
        L.check(self.h, self._ordered(self.lib.hdg_trace_apply_dev, L._ptr(x), L._ptr(y)))

    def condensed_rhs_dev(self, r_u, r_h, g) -> None:
        L.check(self.h, self._ordered(self.lib.hdg_condensed_rhs_dev, L._ptr(r_u), L._ptr(r_h), L._ptr(g)))

    def precond_apply_dev(self, v, z) -> None:
        L.check(self.h, self._ordered(self.lib.hdg_precond_apply_dev, L._ptr(v), L._ptr(z)))

    def precond_apply32_dev(self, v, z) -> None:
        L.check(self.h, self._ordered(self.lib.hdg_precond_apply32_dev, L._ptr(v), L._ptr(z)))

    def autotune(self) -> tuple:
        """Time candidate launch shapes on this handle and keep the fastest;
        returns (threads per facet-row block, Gram-Schmidt blocks, largest
        single-CTA coarse level)."""
        ch = np.zeros(3, dtype=np.int32)
        L.check(self.h, self.lib.hdg_autotune(self.h, ch.ctypes.data))
        return tuple(int(v) for v in ch)

    # ---------------------------------------------------------------- learned smoother
    def learned_init(self, hidden: int = 32, capacity: int = 256, seed: int = 0) -> int:
        n = C.c_int32()
        L.check(self.h, self.lib.hdg_learned_init(self.h, int(hidden), int(capacity), C.c_uint64(seed), C.byref(n)))
        self.n_learned_params = int(n.value)
        return self.n_learned_params

    def learned_collect_dev(self, r_u, r_h) -> int:
        n = C.c_int32()
        L.check(self.h, self._ordered(self.lib.hdg_learned_collect_dev, L._ptr(r_u), L._ptr(r_h), C.byref(n)))
        return int(n.value)

    def learned_train(self, steps: int, batch: int = 8, lr: float = 1e-3):
        a, b = C.c_double(), C.c_double()
        L.check(self.h, self.lib.hdg_learned_train(self.h, int(steps), int(batch), C.c_double(lr), C.byref(a),
                                                   C.byref(b)))
        return a.value, b.value

    def learned_params(self) -> np.ndarray:
        th = np.empty(self.n_learned_params, dtype=np.float32)
        L.check(self.h, self.lib.hdg_learned_params(self.h, th.ctypes.data, 1))
        return th

    def set_learned_params(self, theta) -> None:
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.n_learned_params
        L.check(self.h, self.lib.hdg_learned_params(self.h, th.ctypes.data, 0))

    def learned_enable(self, on: bool = True, tensor_cores: bool = False) -> None:
        """Use the learned sweep in later solves; tensor_cores runs its network
        as BF16 tcgen05 GEMMs (FP32 accumulation) instead of FP32 on the CUDA cores."""
        L.check(self.h, self.lib.hdg_learned_enable(self.h, (2 if tensor_cores else 1) if on else 0))

    def learned_loss_grad_dev(self, R):
        """R: float32 device tensor [n, n_facets, p+1]; returns (loss, gradient)."""
        g = np.empty(self.n_learned_params, dtype=np.float32)
        loss = C.c_double()
        L.check(self.h, self._ordered(self.lib.hdg_learned_loss_grad_dev, L._ptr(R), int(R.shape[0]), g.ctypes.data,
                                      C.byref(loss)))
        return loss.value, g

    def chebyshev(self, coarse: bool = False):
        """The Chebyshev smoother's ellipse (theta, delta^2) and the Ritz values it was
        fitted to; coarse=True: those of the Lax-Friedrichs RT0 coarse solve."""
        ell = np.zeros(2)
        ritz = np.zeros(128)
        n = C.c_int32(0)
        fn = self.lib.hdg_get_rt0_chebyshev if coarse else self.lib.hdg_get_chebyshev
        L.check(self.h, fn(self.h, ell.ctypes.data, ritz.ctypes.data, C.byref(n)))
        return (float(ell[0]), float(ell[1])), ritz[:2 * n.value:2] + 1j * ritz[1:2 * n.value:2]

    # ---------------------------------------------------------------- IMEX time stepping
    def imex_init(self, f_vertex=None) -> None:
        """Explicit Coriolis field (host, [n_vertices]) for hdg_imex_step_dev."""
        fv = None if f_vertex is None else np.ascontiguousarray(f_vertex, dtype=np.float64)
        L.check(self.h, self.lib.hdg_imex_init(self.h, None if fv is None else fv.ctypes.data))

    def imex_rates_dev(self, u, h, nu, nh, lu, lh) -> None:
        """(nu, nh) = M^-1 N(q) (both None to skip), (lu, lh) = M^-1 L(q)."""
        L.check(self.h, self._ordered(self.lib.hdg_imex_rates_dev, L._ptr(u), L._ptr(h), L._ptr(nu), L._ptr(nh),
                                      L._ptr(lu), L._ptr(lh)))

    def imex_step_dev(self, scheme, dt: float, u, h, theta: float = 0.5, allow_fail: bool = False) -> dict:
        """One step of an IMEX scheme ("theta", "ARS2", "SSP2", "ARS3") on device (u, h), in place."""
        info = L.hdg_solve_info()
        code = L.IMEX_SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        rc = self._ordered(self.lib.hdg_imex_step_dev, code, C.c_double(theta), C.c_double(dt), L._ptr(u), L._ptr(h),
                           C.byref(info))
        L.check(self.h, rc, allow=(L.HDG_ENOCONV, L.HDG_EBREAKDOWN) if allow_fail else ())
        return info.as_dict()

    # ---------------------------------------------------------------- accounting
    def profile_enable(self, timing: bool = True, cold: bool = False) -> None:
        """Launch counts always; with timing, per-category CUDA-event times; with
        cold, the L2 cache is evicted before every timed launch."""
        L.check(self.h, self.lib.hdg_profile_enable(self.h, (2 if cold else 1) if timing else 0))

    def profile_read(self) -> dict:
        ms = np.zeros(L.HDG_PROF_N)
        n = np.zeros(L.HDG_PROF_N, dtype=np.int64)
        L.check(self.h, self.lib.hdg_profile_read(self.h, ms.ctypes.data, n.ctypes.data))
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(L.PROF_NAMES)}

    # ---------------------------------------------------------------- inspection
    def facets(self):
        fo = np.empty((self.n_cells, 3), np.int32)
        fl = np.empty((self.n_cells, 3), np.int32)
        fv = np.empty((self.n_facets, 2), np.int32)
        L.check(self.h, self.lib.hdg_get_facets(self.h, fo.ctypes.data, fl.ctypes.data, fv.ctypes.data))
        return fo, fl, fv

    def cell_schur(self) -> np.ndarray:
        S = np.empty((self.n_cells, self.m, self.m))
        L.check(self.h, self.lib.hdg_get_cell_schur(self.h, S.ctypes.data))
        return S


def solve_batch_dev(solvers, r_u, r_h, lam, n_threads: int = 0, allow_fail: bool = False):
    """Run independent solves concurrently (``hdg_solve_batch_dev``): solver i
    solves device tensors ``r_u[i], r_h[i]`` into ``lam[i]``.  Every solver
    needs its own stream (the default).  Returns the list of info dicts."""
    lib = L.load()
    n = len(solvers)
    torch = _torch()
    if torch is not None:
        cur = torch.cuda.current_stream()
        for s in solvers:
            s.stream.wait_stream(cur)
    hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
    pu = (C.c_void_p * n)(*[L._ptr(t) for t in r_u])
    ph = (C.c_void_p * n)(*[L._ptr(t) for t in r_h])
    pl = (C.c_void_p * n)(*[L._ptr(t) for t in lam])
    infos = (L.hdg_solve_info * n)()
    rc = lib.hdg_solve_batch_dev(hs, n, pu, ph, pl, infos, int(n_threads))
    if torch is not None:
        for s in solvers:
            cur.wait_stream(s.stream)
    if rc != 0 and not (allow_fail and rc in (L.HDG_ENOCONV, L.HDG_EBREAKDOWN)):
        raise L.HDGError(rc, (lib.hdg_last_error(None) or b"").decode())
    return [infos[i].as_dict() for i in range(n)]


class MergedBatch:
    """Merged batched solves (``hdg_batch_*``): one host thread drives the
    solves of every solver, whose launches run as merged multi-problem
    kernels in one CUDA graph per wave.  Solvers must use the precision
    HDG_MIXED_FP32 or HDG_MIXED_BF16 (upwind flux, reorth = 0).  Close the
    batch before its solvers."""

    def __init__(self, solvers):
        self.lib = L.load()
        self.solvers = list(solvers)
        n = len(self.solvers)
        hs = (C.c_void_p * n)(*[s.h.value for s in self.solvers])
        self.b = C.c_void_p()
        L.check(None, self.lib.hdg_batch_create(hs, n, C.byref(self.b)))

    def solve_dev(self, r_u, r_h, lam, allow_fail: bool = False):
        """Solver i solves device tensors ``r_u[i], r_h[i]`` into ``lam[i]``
        (complete on return).  Returns the list of info dicts."""
        n = len(self.solvers)
        torch = _torch()
        if torch is not None:
            cur = torch.cuda.current_stream()
            for s in self.solvers:
                s.stream.wait_stream(cur)
        pu = (C.c_void_p * n)(*[L._ptr(t) for t in r_u])
        ph = (C.c_void_p * n)(*[L._ptr(t) for t in r_h])
        pl = (C.c_void_p * n)(*[L._ptr(t) for t in lam])
        infos = (L.hdg_solve_info * n)()
        rc = self.lib.hdg_batch_solve_dev(self.b, pu, ph, pl, infos)
        if torch is not None:
            for s in self.solvers:
                cur.wait_stream(s.stream)
        if rc != 0 and not (allow_fail and rc in (L.HDG_ENOCONV, L.HDG_EBREAKDOWN)):
            raise L.HDGError(rc, (self.lib.hdg_last_error(None) or b"").decode())
        return [infos[i].as_dict() for i in range(n)]

    def solve(self, r_u, r_h, allow_fail: bool = False):
        """Host arrays: solver i solves ``r_u[i]`` ([n_cells][2][n_p]), ``r_h[i]``
        ([n_cells][n_p]); returns (list of lambda arrays [n_facets][p+1], infos)."""
        n = len(self.solvers)
        ru = [np.ascontiguousarray(a, dtype=np.float64) for a in r_u]
        rh = [np.ascontiguousarray(a, dtype=np.float64) for a in r_h]
        lam = [np.empty((s.n_facets, s.p + 1)) for s in self.solvers]
        pu = (C.c_void_p * n)(*[a.ctypes.data for a in ru])
        ph = (C.c_void_p * n)(*[a.ctypes.data for a in rh])
        pl = (C.c_void_p * n)(*[a.ctypes.data for a in lam])
        infos = (L.hdg_solve_info * n)()
        rc = self.lib.hdg_batch_solve(self.b, pu, ph, pl, infos)
        if rc != 0 and not (allow_fail and rc in (L.HDG_ENOCONV, L.HDG_EBREAKDOWN)):
            raise L.HDGError(rc, (self.lib.hdg_last_error(None) or b"").decode())
        return lam, [infos[i].as_dict() for i in range(n)]

    def stats(self) -> dict:
        """Waves, merged launches, per-problem launches they carried, graphs
        replayed and graphs built since creation; host nanoseconds spent
        running the problems' host logic, merging/launching waves, and waiting
        for the last waves."""
        a = (C.c_int64 * 8)()
        L.check(None, self.lib.hdg_batch_stats(self.b, a))
        return dict(zip(("waves", "launches", "records", "replays", "builds", "host_ns_fibers", "host_ns_launch",
                         "host_ns_wait"), list(a)))

    def close(self):
        if self.b:
            self.lib.hdg_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
