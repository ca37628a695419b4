"""Independent Crouzeix–Raviart assembly on tetrahedra for Theorem 3.1 in 3D (oracle).

TEST INFRASTRUCTURE ONLY.

The pressure-robust CR scheme of eq. equivCRstWeak with the augmented-Lagrangian
term (eq. k0-stOptEq-ALU), d = 3:
  ν(∇u, ∇v) + β(Π^RT u, Π^RT v) + ε⁻¹(div u, div v),   load (f, Π^RT v).
CR unknowns: the three Cartesian components of the value at every interior face
barycentre.  Local basis on a cell: ψ_i = 1 − 3λ_i (value 1 at the barycentre of
the face opposite vertex i, 0 at the other three).  Π^RT keeps the face fluxes:
∫_{F_i} v·n = |F_i| v_i·n_i, and the RT0 function with unit outward flux on F_i is
(x − x_i)/(3|K|).  Π^CR maps the lowest-order HDG unknowns of a face (normal moment
and the t1, t2 coefficients, all against ℓ_0 = |F|^(-1/2)) to the barycentre value
(c_n n_F + c_1 t1 + c_2 t2)/sqrt|F|.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import tetrahedron_points
from .topology3d import Topology3D


def bary_3d(X, x):
    """Barycentric coordinates (n, 4) of points x (n, 3) in the tetrahedron X (4, 3)."""
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    l = np.linalg.solve(J, (np.atleast_2d(x) - X[0]).T).T
    return np.concatenate([1 - l.sum(axis=1, keepdims=True), l], axis=1)


def cr_cell_3d(X, nu, beta, eps_inv, fvals=None):
    """CR element matrix (12×12, unknown order (i, comp)) and load on one tetrahedron."""
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    Ji = np.linalg.inv(J)
    G = np.concatenate([-Ji.sum(axis=0, keepdims=True), Ji])    # ∇λ_i, (4, 3)
    vol = abs(np.linalg.det(J)) / 6.0
    dpsi = -3.0 * G
    K = np.zeros((12, 12))
    for i in range(4):
        for j in range(4):
            K[3 * i:3 * i + 3, 3 * j:3 * j + 3] += nu * vol * (dpsi[i] @ dpsi[j]) * np.eye(3)
    dv = dpsi.reshape(-1)                     # div v = Σ_i v_i · ∇ψ_i
    K += eps_inv * vol * np.outer(dv, dv)
    xq, wq = tetrahedron_points(X, 3)
    PRT = np.zeros((xq.shape[0], 12, 3))
    for i in range(4):
        o = [j for j in range(4) if j != i]
        cr = np.cross(X[o[1]] - X[o[0]], X[o[2]] - X[o[0]])
        area = 0.5 * np.linalg.norm(cr)
        n = cr / np.linalg.norm(cr)
        if n @ (X[o[0]] - X[i]) < 0:
            n = -n
        phi = (xq - X[i]) / (3.0 * vol)
        for c in range(3):
            PRT[:, 3 * i + c, :] += area * n[c] * phi
    K += beta * np.einsum("q,qic,qjc->ij", wq, PRT, PRT)
    F = None
    if fvals is not None:
        fq = bary_3d(X, xq) @ np.asarray(fvals).reshape(4, 3)   # linear f from its vertex values
        F = np.einsum("q,qc,qic->i", wq, fq, PRT)
    return K, F


def cr_system_3d(topo: Topology3D, nu, beta, eps_inv, fvals=None):
    """Global CR matrix (3 n_int × 3 n_int) and load; unknown 3i+c ↔ face i, component c."""
    n = 3 * topo.n_interior
    rows, cols, vals = [], [], []
    F = np.zeros(n)
    for c in range(topo.n_cells):
        Kc, Fc = cr_cell_3d(topo.coords[topo.cells[c]], nu, beta, eps_inv,
                            None if fvals is None else fvals[c])
        idx = -np.ones(12, dtype=np.int64)
        for i in range(4):
            ii = topo.interior_index[topo.cell_facets[c, i]]
            if ii >= 0:
                idx[3 * i:3 * i + 3] = 3 * ii + np.arange(3)
        m = idx >= 0
        I = idx[m]
        rows.append(np.repeat(I, len(I)))
        cols.append(np.tile(I, len(I)))
        vals.append(Kc[np.ix_(m, m)].ravel())
        if Fc is not None:
            F[I] += Fc[m]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A, F


def pi_cr_matrix_3d(topo: Topology3D) -> sp.csr_matrix:
    """Π^CR: lowest-order HDG unknowns (3 per interior face) -> CR barycentre values."""
    rows, cols, vals = [], [], []
    for i, F in enumerate(topo.interior_facets):
        _, _, _, area, t1, t2, nF = topo.facet_geometry(F)
        for c in range(3):
            for a, v in enumerate((nF, t1, t2)):
                rows.append(3 * i + c)
                cols.append(3 * i + a)
                vals.append(v[c] / np.sqrt(area))
    n = 3 * topo.n_interior
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
