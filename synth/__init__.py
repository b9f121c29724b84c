"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds mesh and right-hand-side generators only: vertex positions,
triangle lists, Dirichlet masks and random vectors.  It contains none of the
solver's arithmetic (no Laplacian, mass matrix, prolongation or cycle), so the
oracle and the CUDA path can both consume its output without sharing method code.
"""
from .meshes import (icosahedron, icosphere, perturbed_icosphere, geodesic_sphere,
                     perturbed_geodesic_sphere,
                     torus, disk, sh_noise, mean_edge_length, boundary_mask,
                     euler_characteristic, sinusoidal_displacement)
from .rhs import uniform_rhs, unit_directions

__all__ = ["icosahedron", "icosphere", "perturbed_icosphere", "geodesic_sphere",
           "perturbed_geodesic_sphere",
           "torus", "disk", "sh_noise", "mean_edge_length", "boundary_mask",
           "euler_characteristic", "sinusoidal_displacement", "uniform_rhs", "unit_directions"]
