"""Triangle meshes used as synthetic inputs.

Two families, matching the grids of the paper's experiments:

* the doubly periodic square of Sec. 7.1 ("Grid layout"): ``n x n`` squares of
  side ``L/n``, each cut into two triangles, ``N = 2 n^2`` cells
  (Tab. grid_setup);
* the icosahedral sphere of Sec. 7.9: the 20 faces of an icosahedron refined
  ``r`` times by edge midpoints pushed back onto the sphere,
  ``N = 20 * 4^r`` cells, average edge ``h = 2^-r h_0 R`` with
  ``h_0 = sqrt(4 pi / (5 sqrt 3))`` (Tab. grid_setup_spherical).

Conventions of the arrays (they are the input layout of the library):

* ``cell_vertices[K] = (v0, v1, v2)`` is counter-clockwise (seen from outside
  on the sphere);
* on the periodic square ``vertex_xyz`` holds the wrapped coordinates in
  ``[0, L)^2`` and ``cell_shift[K, i]`` the offset (0 or +-L per component) that
  unwraps vertex ``i`` of cell ``K`` so the cell is a proper triangle;
* coarse levels are produced by the same generators at coarser resolution;
  ``level.parent[i] = (a, b)`` says that vertex ``i`` of the next *finer*
  level sits at the midpoint of coarse vertices ``a`` and ``b`` (``a == b``
  for a vertex that exists on both levels).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Mesh:
    dim: int                          # 2: flat periodic square, 3: sphere
    vertex_xyz: np.ndarray            # float64 [n_vertices, dim]
    cell_vertices: np.ndarray         # int32 [n_cells, 3], counter-clockwise
    cell_shift: np.ndarray | None     # float64 [n_cells, 3, 2] (flat) or None
    radius: float                     # sphere radius, 0 for flat
    h: float                          # nominal mesh size used for Courant numbers
    side: float = 0.0                 # side length of the periodic square (flat)
    parent: np.ndarray | None = None  # int32 [n_vertices of next finer level, 2]
    levels: list = field(default_factory=list)  # coarser levels, next-coarser first
    name: str = ""

    @property
    def n_cells(self) -> int:
        return int(self.cell_vertices.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.vertex_xyz.shape[0])

    def cell_coords(self) -> np.ndarray:
        """Unwrapped vertex coordinates per cell, float64 [n_cells, 3, dim]."""
        x = self.vertex_xyz[self.cell_vertices]
        if self.cell_shift is not None:
            x = x + self.cell_shift
        return x


# --------------------------------------------------------------------------
# doubly periodic square
# --------------------------------------------------------------------------

def periodic_square(n: int, side: float = 1.0) -> Mesh:
    """``n x n`` periodic squares, each split along its (i,j)-(i+1,j+1) diagonal.

    Vertex ``(i, j)`` has id ``j*n + i``; square ``s = j*n + i`` owns cells
    ``2s`` (below the diagonal) and ``2s+1`` (above it).
    """
    if n < 3:
        raise ValueError("periodic square needs n >= 3 (smaller grids repeat facets)")
    hs = side / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    xyz = np.stack([ii.ravel() * hs, jj.ravel() * hs], axis=1).astype(np.float64)

    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    shift = np.zeros((2 * n * n, 3, 2), dtype=np.float64)
    for j in range(n):
        for i in range(n):
            s = j * n + i
            ip, jp = (i + 1) % n, (j + 1) % n
            sx = side if i + 1 == n else 0.0
            sy = side if j + 1 == n else 0.0
            v00, v10, v11, v01 = j * n + i, j * n + ip, jp * n + ip, jp * n + i
            cells[2 * s] = (v00, v10, v11)
            shift[2 * s] = ((0, 0), (sx, 0), (sx, sy))
            cells[2 * s + 1] = (v00, v11, v01)
            shift[2 * s + 1] = ((0, 0), (sx, sy), (0, sy))
    return Mesh(dim=2, vertex_xyz=xyz, cell_vertices=cells, cell_shift=shift,
                radius=0.0, h=hs, side=side, name=f"square{n}")


def _square_parent(n_fine: int) -> np.ndarray:
    """Parents (on the n_fine/2 grid) of each vertex of the n_fine grid."""
    nc = n_fine // 2
    par = np.empty((n_fine * n_fine, 2), dtype=np.int32)
    for J in range(n_fine):
        for I in range(n_fine):
            a = ((J // 2) % nc) * nc + (I // 2) % nc
            if I % 2 == 0 and J % 2 == 0:
                b = a
            else:
                # odd index: neighbour one coarse step further along that axis
                I2 = (I // 2 + (I % 2)) % nc
                J2 = (J // 2 + (J % 2)) % nc
                b = J2 * nc + I2
            par[J * n_fine + I] = (a, b)
    return par


def periodic_square_hierarchy(n: int, side: float = 1.0, n_coarsest: int = 4) -> Mesh:
    """Fine periodic square plus its coarse levels ``n/2, n/4, ..., n_coarsest``.

    Each coarse level is the periodic square at half the resolution; the
    fine mesh is its uniform midpoint refinement (nested P1 spaces).
    """
    fine = periodic_square(n, side)
    levels = []
    nf = n
    while nf // 2 >= max(n_coarsest, 3) and nf % 2 == 0:
        lev = periodic_square(nf // 2, side)
        lev.parent = _square_parent(nf)
        levels.append(lev)
        nf //= 2
    fine.levels = levels
    return fine


# --------------------------------------------------------------------------
# icosahedral sphere
# --------------------------------------------------------------------------

def _icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """Unit icosahedron: the 12 cyclic permutations of (0, +-1, +-phi).

    Faces are found as the vertex triples that are pairwise at the edge
    length 2, then oriented counter-clockwise seen from outside.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts.append((0.0, s1, s2 * phi))
            pts.append((s1, s2 * phi, 0.0))
            pts.append((s2 * phi, 0.0, s1))
    v = np.array(pts, dtype=np.float64)
    nv = len(v)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    for a in range(nv):
        for b in range(a + 1, nv):
            if not adj[a, b]:
                continue
            for c in range(b + 1, nv):
                if adj[a, c] and adj[b, c]:
                    if np.dot(np.cross(v[b] - v[a], v[c] - v[a]), v[a]) > 0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    f = np.array(faces, dtype=np.int32)
    assert f.shape == (20, 3)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def _refine_sphere(v: np.ndarray, f: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """One midpoint refinement; new vertices are appended and normalised."""
    nv = len(v)
    mid: dict[tuple[int, int], int] = {}
    newv = []
    parent = [(i, i) for i in range(nv)]

    def midpoint(a: int, b: int) -> int:
        key = (a, b) if a < b else (b, a)
        if key not in mid:
            mid[key] = nv + len(newv)
            m = v[a] + v[b]
            newv.append(m / np.linalg.norm(m))
            parent.append(key)
        return mid[key]

    cells = np.empty((4 * len(f), 3), dtype=np.int32)
    for k, (a, b, c) in enumerate(f):
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        cells[4 * k + 0] = (a, ab, ca)
        cells[4 * k + 1] = (ab, b, bc)
        cells[4 * k + 2] = (ca, bc, c)
        cells[4 * k + 3] = (ab, bc, ca)
    vv = np.concatenate([v, np.array(newv)], axis=0)
    return vv, cells, np.array(parent, dtype=np.int32)


H0_SPHERE = math.sqrt(4.0 * math.pi / (5.0 * math.sqrt(3.0)))


def _sphere_levels(r: int, radius: float):
    v, f = _icosahedron()
    out = [(v, f, None)]
    for _ in range(r):
        v, f, par = _refine_sphere(v, f)
        out.append((v, f, par))
    meshes = []
    for lev, (vv, ff, _) in enumerate(out):
        meshes.append(Mesh(dim=3, vertex_xyz=vv * radius, cell_vertices=ff.copy(),
                           cell_shift=None, radius=radius,
                           h=(2.0 ** -lev) * H0_SPHERE * radius, name=f"sphere_r{lev}"))
    # parent of level l+1 vertices, stored on level l
    for lev in range(r):
        meshes[lev].parent = out[lev + 1][2]
    return meshes


def icosahedral_sphere(r: int, radius: float = 1.0) -> Mesh:
    """Icosahedral sphere at refinement ``r`` (``20*4^r`` cells), no coarse levels."""
    return _sphere_levels(r, radius)[-1]


def sphere_hierarchy(r: int, radius: float = 1.0, r_coarsest: int = 1) -> Mesh:
    """Sphere at refinement ``r`` with coarse levels ``r-1, ..., r_coarsest``."""
    ms = _sphere_levels(r, radius)
    fine = ms[-1]
    fine.levels = [ms[lev] for lev in range(r - 1, max(r_coarsest, 0) - 1, -1)]
    return fine
