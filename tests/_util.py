"""Small shared helpers for the CPU tests (mesh → oracle objects)."""
import numpy as np

from workloads import unit_square, unit_square_hierarchy, forcing_at_lattice
from oracle.topology import build_topology


def topo_of(mesh):
    return build_topology(mesh.coords, mesh.cells, mesh.vertex_colour)


def hierarchy(N0, n_levels, **kw):
    ms = unit_square_hierarchy(N0, n_levels, **kw)
    return ms, [topo_of(m) for m in ms], [m.parent for m in ms]


def forcing(mesh, k, sol, nu, beta):
    return forcing_at_lattice(mesh.coords, mesh.cells, k, sol.forcing(nu, beta))


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
