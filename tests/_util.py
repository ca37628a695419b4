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


def parity_opts(hdg, gamma):
    """Solve options for the FP64 parity target against the exact discrete solution:
    inner relative 1e-10, Uzawa pressure-error estimate 1e-11, and a residual floor of
    1e-12 |F| where FP64 reaches it.  At gamma = 1e4 the augmented-Lagrangian term makes
    residuals below about 1e-10 |F| round-off (Remark 3.1), so the floor stays there."""
    o = hdg.default_solve_opts()
    o.rtol, o.uzawa_tol = 1e-10, 1e-11
    o.floor_rel = 1e-12 if gamma <= 1e2 else 1e-10
    return o


def relnorm(a, b):
    """2-norm relative error |a - b| / |b|."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
