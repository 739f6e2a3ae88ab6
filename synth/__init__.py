"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no finite-element arithmetic: it only produces meshes (vertex
coordinates and cell connectivity) and random vectors.  The oracle and the CUDA
library each derive everything else (quadrature, basis, DoF numbering, geometry)
on their own.
"""
from .mesh import curved_nodes, kuhn_cube, shuffle_mesh, jitter_interior
from .vectors import uniform_vector, lognormal_coefficients, SEEDS

__all__ = [
    "kuhn_cube",
    "shuffle_mesh",
    "jitter_interior",
    "curved_nodes",
    "uniform_vector",
    "lognormal_coefficients",
    "SEEDS",
]
