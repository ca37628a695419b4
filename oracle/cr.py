"""Independent Crouzeix–Raviart assembly for Theorem 3.1 (oracle).

TEST INFRASTRUCTURE ONLY.

The pressure-robust CR scheme of eq. equivCRstWeak, with the augmented
Lagrangian term of the lowest-order operator (eq. k0-stOptEq-ALU):
  ν(∇u, ∇v) + β(Π^RT u, Π^RT v) + ε⁻¹(div u, div v),   load (f, Π^RT v).
CR unknowns: the two Cartesian components of the value at every interior
facet midpoint.  Local basis on a cell: ψ_i = 1 − 2λ_i (value 1 at the
midpoint of the facet opposite vertex i, 0 at the other two midpoints).

Π^RT (eq. CR_2RT0) keeps the facet fluxes: for v = Σ v_i ψ_i on K,
∫_{F_i} v·n = |F_i| v_i·n_i, and the RT0 function with unit outward flux on
F_i is (x − x_i)/(2|K|).  Π^CR (eq. RT0N1_2CR) maps the lowest-order HDG
unknowns of a facet (normal moment c_n, tangential coefficient c_t, both
against ℓ_0 = |F|^{-1/2}) to the midpoint value (c_n n_F + c_t t_F)/sqrt|F|.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads.manufactured import lattice_barycentric_2d

from .quadrature import triangle_points
from .topology import Topology


def _bary_grads(X):
    J = np.stack([X[1] - X[0], X[2] - X[0]], axis=1)
    Jinv = np.linalg.inv(J)
    g1, g2 = Jinv[0], Jinv[1]
    return np.stack([-g1 - g2, g1, g2]), 0.5 * abs(np.linalg.det(J))


def _bary(X, x):
    J = np.stack([X[1] - X[0], X[2] - X[0]], axis=1)
    l12 = np.linalg.solve(J, (x - X[0]).T).T
    return np.stack([1 - l12[:, 0] - l12[:, 1], l12[:, 0], l12[:, 1]], axis=1)


def cr_cell(X, nu, beta, eps_inv, fvals=None):
    """CR element matrix (6×6, unknown order (i, comp)) and load on one cell."""
    G, area = _bary_grads(X)
    dpsi = -2.0 * G                                   # ∇ψ_i
    K = np.zeros((6, 6))
    for i in range(3):
        for j in range(3):
            K[2 * i:2 * i + 2, 2 * j:2 * j + 2] += nu * area * (dpsi[i] @ dpsi[j]) * np.eye(2)
    # div v = Σ_i v_i · ∇ψ_i (constant on K)
    dv = np.zeros(6)
    for i in range(3):
        dv[2 * i:2 * i + 2] = dpsi[i]
    K += eps_inv * area * np.outer(dv, dv)
    # Π^RT: coefficient of RT0 function i = |F_i| v_i·n_i
    xq, wq = triangle_points(X, 3)
    PRT = np.zeros((xq.shape[0], 6, 2))   # values of Π^RT(ψ_i e_c) at xq
    for i in range(3):
        a, b = [j for j in range(3) if j != i]
        e = X[b] - X[a]
        Fi = np.hypot(*e)
        n = np.array([e[1], -e[0]]) / Fi
        if n @ (0.5 * (X[a] + X[b]) - X[i]) < 0:
            n = -n
        phi = (xq - X[i]) / (2 * area)
        for c in range(2):
            PRT[:, 2 * i + c, :] += Fi * n[c] * phi
    K += beta * np.einsum("q,qic,qjc->ij", wq, PRT, PRT)
    F = None
    if fvals is not None:
        lam = lattice_barycentric_2d(1)             # degree-1 lattice = vertices
        Xl = lam @ X
        # f_h is linear: evaluate by barycentric interpolation of the lattice values
        bl = _bary(X, Xl)
        coef = np.linalg.solve(bl, np.asarray(fvals).reshape(-1, 2))   # values at vertices
        fq = _bary(X, xq) @ coef
        F = np.einsum("q,qc,qic->i", wq, fq, PRT)
    return K, F


def cr_system(topo: Topology, nu, beta, eps_inv, fvals=None):
    """Global CR matrix (2 n_int × 2 n_int) and load; unknown 2i+c ↔ facet i, component c."""
    n = 2 * topo.n_interior
    rows, cols, vals = [], [], []
    F = np.zeros(n)
    for c in range(topo.n_cells):
        X = topo.coords[topo.cells[c]]
        Kc, Fc = cr_cell(X, nu, beta, eps_inv, None if fvals is None else fvals[c])
        idx = -np.ones(6, dtype=np.int64)
        for i in range(3):
            ii = topo.interior_index[topo.cell_facets[c, i]]
            if ii >= 0:
                idx[2 * i:2 * i + 2] = 2 * ii + np.arange(2)
        m = idx >= 0
        I = idx[m]
        rows.append(np.repeat(I, len(I)))
        cols.append(np.tile(I, len(I)))
        vals.append(Kc[np.ix_(m, m)].ravel())
        if Fc is not None:
            F[I] += Fc[m]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return A, F


def pi_cr_matrix(topo: Topology) -> sp.csr_matrix:
    """Π^CR: lowest-order HDG unknowns (2 per interior facet) -> CR midpoint values."""
    n = topo.n_interior
    rows, cols, vals = [], [], []
    for i, F in enumerate(topo.interior_facets):
        _, _, L, t, nF = topo.facet_geometry(F)
        for c in range(2):
            rows += [2 * i + c, 2 * i + c]
            cols += [2 * i, 2 * i + 1]
            vals += [nF[c] / np.sqrt(L), t[c] / np.sqrt(L)]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
