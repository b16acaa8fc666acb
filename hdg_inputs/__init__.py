"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package only *generates data*: triangle meshes (doubly periodic squares,
icosahedral spheres) with their nested coarse levels, Coriolis values at the
vertices and right-hand-side fields sampled at the nodes of the DG layout.  It
holds none of the discretisation's arithmetic (no bases, no integrals, no
local matrices, no solver); the oracle and the CUDA library each build those
on their own from the mesh arrays produced here.
"""
from .meshes import (Mesh, periodic_square, icosahedral_sphere,
                     periodic_square_hierarchy, sphere_hierarchy)
from .fields import (dg_node_positions, cell_frames, manufactured_rhs,
                     gaussian_field_rhs, spherical_harmonic_rhs, add_noise,
                     coriolis_flat, coriolis_sphere)

__all__ = [
    "Mesh", "periodic_square", "icosahedral_sphere", "periodic_square_hierarchy",
    "sphere_hierarchy", "dg_node_positions", "cell_frames", "manufactured_rhs",
    "gaussian_field_rhs", "spherical_harmonic_rhs", "add_noise",
    "coriolis_flat", "coriolis_sphere",
]
