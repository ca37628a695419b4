"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds only input generation: structured simplicial meshes and
their refinement hierarchy, the manufactured solutions of the generalized
Stokes problem (Section 3.1, eq. stModel) evaluated in closed form, forcing
values sampled at the element lattice points that the library's input format
expects, and seeded random vectors.  It contains none of the discretisation
or solver arithmetic: neither the oracle nor the CUDA library is imported here,
and the package imports neither of them.
"""

from .mesh2d import unit_square, unit_square_hierarchy, Mesh2D
from .manufactured import (curl_bubble_2d, polynomial_2d, forcing_at_lattice,
                           lattice_points_2d, n_lattice_2d)

__all__ = ["unit_square", "unit_square_hierarchy", "Mesh2D",
           "curl_bubble_2d", "polynomial_2d", "forcing_at_lattice",
           "lattice_points_2d", "n_lattice_2d"]
