"""Seeded synthetic inputs for the particle-location path.

This package is the one place both sides read their inputs from: the CUDA
path under test and the CPU oracle. It holds no arithmetic of the method
itself (no barycentric coordinates, no neighbour search, no walk): only
meshes (coordinates + connectivity), analytic velocity fields sampled at
the mesh nodes, and the time step that gives a requested CFL number.

The workloads stand in for the paper's lid-driven cavity and flow-past-a-
sphere meshes (Sec. 3), which need the external L-G solver and are not
available: a jittered, Delaunay-triangulated unit square (2-D) and a
jittered unit cube split into six Kuhn tetrahedra per lattice cell (3-D).
"""

from .meshes import lattice_2d, delaunay_2d, kuhn_3d, mesh_2d, mesh_3d
from .fields import (rotation, taylor_green, abc_flow, fourier_modes_2d,
                     fourier_modes_3d, dt_for_cfl, cfl_of)
from .cases import make_case, Case, element_node_particles

__all__ = [
    "lattice_2d", "delaunay_2d", "kuhn_3d", "mesh_2d", "mesh_3d",
    "rotation", "taylor_green", "abc_flow", "fourier_modes_2d",
    "fourier_modes_3d", "dt_for_cfl", "cfl_of", "make_case", "Case", "element_node_particles",
]
