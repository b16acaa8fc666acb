"""Argument and mesh validation in hdg_setup, on the CPU: every check runs on the host
before the first CUDA call, so each malformed input is rejected with
HDG_EINVAL, no handle and a message naming the fault, without a GPU."""
import copy
import ctypes

import numpy as np
import pytest

import hdg_inputs as I


def _setup(mesh, p=1):
    """hdg_setup on mesh (a mesh object, or None for a NULL descriptor)."""
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    prm = _lib.default_params()
    prm.p = p
    prm.tau, prm.g, prm.H = 0.1, 1.0, 1.0
    keep = []
    desc = None if mesh is None else _lib.make_mesh_desc(mesh, keep)
    h = ctypes.c_void_p()
    rc = lib.hdg_setup(None if desc is None else ctypes.byref(desc), ctypes.byref(prm), None, ctypes.byref(h))
    return rc, h.value, lib.hdg_last_error(None).decode()


def _mesh():
    return I.periodic_square_hierarchy(8, n_coarsest=2)      # 64 vertices, one coarse level of 16


def _flip_one_cell(m):
    m.cell_vertices = m.cell_vertices.copy()
    m.cell_vertices[0, [1, 2]] = m.cell_vertices[0, [2, 1]]
    m.cell_shift = m.cell_shift.copy()
    m.cell_shift[0, [1, 2]] = m.cell_shift[0, [2, 1]]


def _case(name):
    m = copy.deepcopy(_mesh())
    if name == "null":
        return None, "mesh descriptor is NULL"
    if name == "empty":
        m.cell_vertices = m.cell_vertices[:0]
        m.cell_shift = m.cell_shift[:0]
        return m, "empty mesh"
    if name == "dim":
        m.dim = 4
        return m, "dim must be 2 or 3"
    if name == "index":
        m.cell_vertices = m.cell_vertices.copy()
        m.cell_vertices[3, 1] = m.n_vertices + 5
        return m, "vertex index out of range"
    if name == "no_shift":
        m.cell_shift = None
        return m, "need cell_shift"
    if name == "open":
        m.cell_vertices = m.cell_vertices[1:]
        m.cell_shift = m.cell_shift[1:]
        return m, "not closed"
    if name == "repeated":
        # vertex 0 of cell 2 again as its third vertex, at a periodic image that
        # keeps the cell counter-clockwise (so that the orientation check passes)
        m.cell_vertices = m.cell_vertices.copy()
        m.cell_shift = m.cell_shift.copy()
        cv, sh, X = m.cell_vertices[2], m.cell_shift[2], m.vertex_xyz
        p0, p1 = X[cv[0]] + sh[0], X[cv[1]] + sh[1]
        for d in ([m.side, 0.0], [0.0, m.side], [-m.side, 0.0], [0.0, -m.side]):
            p2 = X[cv[0]] + sh[0] + np.array(d)
            if (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]) > 0:
                break
        m.cell_vertices[2, 2] = cv[0]
        m.cell_shift[2, 2] = sh[0] + np.array(d)
        return m, "repeated vertex"
    if name == "orientation":
        _flip_one_cell(m)
        return m, "counter-clockwise"
    if name == "non_manifold":
        m.cell_vertices = np.concatenate([m.cell_vertices, m.cell_vertices[:1]])
        m.cell_shift = np.concatenate([m.cell_shift, m.cell_shift[:1]])
        return m, "more than two cells"
    if name == "no_parent":
        m.levels[0].parent = None
        return m, "parent array is NULL"
    if name == "parent_range":
        m.levels[0].parent = m.levels[0].parent.copy()
        m.levels[0].parent[5, 0] = m.levels[0].n_vertices
        return m, "parent index out of range"
    if name == "coarse_dim":
        m.levels[0].dim = 3
        return m, "dim differs"
    if name == "coarsest_too_large":
        return I.periodic_square_hierarchy(48, n_coarsest=48), "more than 1024 vertices"
    sph = copy.deepcopy(I.sphere_hierarchy(2, 1.0, r_coarsest=1))
    if name == "sphere_degenerate":
        sph.cell_vertices = sph.cell_vertices.copy()
        sph.cell_vertices[4, 1] = sph.cell_vertices[4, 0]
        return sph, "degenerate cell"
    if name == "sphere_orientation":
        # a cell listed clockwise seen from outside: locally fine in its own frame,
        # its facets then run the same way as its neighbours'
        sph.cell_vertices = sph.cell_vertices.copy()
        sph.cell_vertices[4, [1, 2]] = sph.cell_vertices[4, [2, 1]]
        return sph, "inconsistent cell orientation"
    raise ValueError(name)


CASES = ["null", "empty", "dim", "index", "no_shift", "open", "repeated", "orientation", "non_manifold",
         "no_parent", "parent_range", "coarse_dim", "coarsest_too_large", "sphere_degenerate", "sphere_orientation"]


@pytest.mark.parametrize("name", CASES)
def test_malformed_mesh_is_rejected_on_the_host(name):
    from paper_2004_09389_gb300 import _lib
    mesh, text = _case(name)
    rc, h, msg = _setup(mesh)
    assert rc == _lib.HDG_EINVAL and not h
    assert text in msg, msg


def test_bad_coarse_level_list_is_rejected_on_the_host():
    """n_coarse > 0 with a NULL level array, and a negative count."""
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    prm = _lib.default_params()
    prm.tau, prm.g, prm.H = 0.1, 1.0, 1.0
    keep = []
    for n_coarse in (1, -1):
        desc = _lib.make_mesh_desc(_mesh(), keep)
        desc.n_coarse = n_coarse
        desc.coarse = None
        h = ctypes.c_void_p()
        rc = lib.hdg_setup(ctypes.byref(desc), ctypes.byref(prm), None, ctypes.byref(h))
        assert rc == _lib.HDG_EINVAL and not h.value
        assert "bad coarse level list" in lib.hdg_last_error(None).decode()


PARAM_FAULTS = [
    ({"p": 0}, "p must be in 1..4"), ({"p": 5}, "p must be in 1..4"),
    ({"tau": 0.0}, "tau, g and H must be positive"), ({"g": -1.0}, "tau, g and H must be positive"),
    ({"H": float("nan")}, "tau, g and H must be positive"),
    ({"rtol": 0.0}, "rtol must be positive"),
    ({"restart": 0}, "restart must be in 1..64"), ({"restart": 65}, "restart must be in 1..64"),
    ({"max_iter": 0}, "max_iter must be positive"),
    ({"n_pre": -1}, "negative sweep count"), ({"p1_nu_post": -2}, "negative sweep count"),
    ({"omega": 0.0}, "damping factors must be positive"), ({"p1_omega": -0.5}, "damping factors must be positive"),
    ({"coarse_mode": 3}, "coarse_mode must be 0, 1 or 2"), ({"coarse_mode": -1}, "coarse_mode must be 0, 1 or 2"),
    ({"smoother": 2}, "smoother must be 0 or 1"),
    ({"smoother": 1, "cheb_steps": 1}, "cheb_steps must be in 2..64"),
    ({"smoother": 1, "cheb_theta": 1.0, "cheb_delta2": 1.5}, "cheb_delta2 must be finite and below cheb_theta^2"),
    ({"reorth": -1}, "reorth must be 0 or 1"),
    ({"precision": 7}, "unknown precision mode"),
    ({"precision": 1, "inner_rtol": 1.0}, "inner_rtol must be in (0, 1)"),
    ({"precision": 2, "inner_rtol": 0.0}, "inner_rtol must be in (0, 1)"),
]


@pytest.mark.parametrize("fields,text", PARAM_FAULTS)
def test_bad_parameters_are_rejected_on_the_host(fields, text):
    """Each parameter fault is reported before the mesh is even looked at."""
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    prm = _lib.default_params()
    prm.tau, prm.g, prm.H = 0.1, 1.0, 1.0
    for k, v in fields.items():
        setattr(prm, k, v)
    keep = []
    desc = _lib.make_mesh_desc(_mesh(), keep)
    h = ctypes.c_void_p()
    rc = lib.hdg_setup(ctypes.byref(desc), ctypes.byref(prm), None, ctypes.byref(h))
    assert rc == _lib.HDG_EINVAL and not h.value
    assert text in lib.hdg_last_error(None).decode()


def test_null_params_and_out_are_rejected():
    from paper_2004_09389_gb300 import _lib
    lib = _lib.load()
    keep = []
    desc = _lib.make_mesh_desc(_mesh(), keep)
    h = ctypes.c_void_p()
    assert lib.hdg_setup(ctypes.byref(desc), None, None, ctypes.byref(h)) == _lib.HDG_EINVAL and not h.value
    assert "params is NULL" in lib.hdg_last_error(None).decode()
    prm = _lib.default_params()
    prm.tau, prm.g, prm.H = 0.1, 1.0, 1.0
    assert lib.hdg_setup(ctypes.byref(desc), ctypes.byref(prm), None, None) == _lib.HDG_EINVAL
    assert "out is NULL" in lib.hdg_last_error(None).decode()
