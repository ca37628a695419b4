"""Objective J = 1/2 ||u_h - u_target||^2 and its adjoint gradients (oracle).

TEST INFRASTRUCTURE ONLY.

The discrete problem is the full H(div)-HDG system of eq. stWeak,
M(nu) X = R(f) with X = (L_h, u_h, û_h, p_h).  For a target field u_target in
[P^{k+1}]^2 (given by its values at each cell's degree-(k+1) lattice),
  dJ/dtheta = lambda^T (dR/dtheta - dM/dtheta X),   M^T lambda = dJ/dX.
For the generalized Stokes system M^T = S M S with S = diag(-I_L, I_u, I_û,
-I_p) (the flux and pressure rows carry the transposed coupling blocks with
opposite signs), so lambda = S M^{-1} (dJ/dX): the adjoint is the primal
problem loaded with the forcing u_h - u_target, and lambda_u = u^a,
lambda_L = -L^a.  The only nu-dependent block is (nu^{-1} L, G)_K, hence
  dJ/dnu_K = nu_K^{-2} (L_h, lambda_L)_K = -nu_K^{-2} (L_h, L^a)_K,
and the forcing enters through (f_h, v)_K, hence
  dJ/df_{K,n,c} = (u^a, lam_n e_c)_K   (lam_n: lattice Lagrange basis).
Both solves are exact (sparse direct) solves of the condensed saddle point.

Oseen (Section 4.1, Picard field w_h fixed): only the (u, û) block gains the
upwind convection C, and S acts as the identity there, so
M^T = S (M_Stokes + C^T) S: the adjoint is the problem whose local
convection block is transposed (HDG(conv_transpose=True)), loaded with
u_h - u_target, with the same two gradient formulas.
"""

from __future__ import annotations

import numpy as np

from workloads.manufactured import lattice_barycentric_2d

from .hdg import HDG
from .quadrature import triangle_points
from .spaces import exponents


def _lattice_values(h: HDG, c: int, coeffs):
    """u_h at the degree-(k+1) lattice of cell c (translated coordinates)."""
    el = h.cells[c].el
    Xl = lattice_barycentric_2d(h.k + 1) @ el.X
    _, u, _, _ = h.fields_at(c, coeffs, Xl)
    return u


def _lattice_function(h: HDG, c: int, vals, xq):
    """Evaluate the [P^{k+1}]^2 field with lattice values `vals` (n_lat, 2) at points xq."""
    cc = h.cells[c]
    return cc.el.mono(xq, h.k + 1) @ (cc.lat_inv @ np.asarray(vals))


def objective_and_gradient(topo, k, fvals, u_target, nu_elem, beta=0.0, gamma=0.0, conv=None):
    """Returns (J, dJ/dfvals (n_cells, n_lat, 2), dJ/dnu (n_cells,), u, p, ua)."""
    h = HDG(topo, k, nu=1.0, beta=beta, gamma=gamma, nu_elem=nu_elem, conv=conv)
    ha = h if conv is None else HDG(topo, k, nu=1.0, beta=beta, gamma=gamma, nu_elem=nu_elem,
                                    conv=conv, conv_transpose=True)
    nc = topo.n_cells
    u, p = h.solve_direct(h.load(fvals))
    prim = [h.recover_cell(c, u, p[c], fvals[c]) for c in range(nc)]
    e = np.stack([_lattice_values(h, c, prim[c]) for c in range(nc)]) - u_target
    J = 0.0
    for c in range(nc):
        xq, wq = triangle_points(h.cells[c].el.X, k + 4)
        ev = _lattice_function(h, c, e[c], xq)
        J += 0.5 * wq @ np.sum(ev ** 2, axis=1)
    ua, pa = ha.solve_direct(ha.load(e))
    gnu = np.zeros(nc)
    gf = np.zeros_like(np.asarray(fvals, dtype=float))
    npk = len(exponents(k))
    for c in range(nc):
        adj = ha.recover_cell(c, ua, pa[c], e[c])
        el = h.cells[c].el
        xq, wq = triangle_points(el.X, k + 4)
        Lp, _, _, _ = h.fields_at(c, prim[c], xq)
        La, uav, _, _ = h.fields_at(c, adj, xq)
        gnu[c] = -np.einsum("q,qij,qij->", wq, Lp, La) / h.nu_elem[c] ** 2
        lam = el.mono(xq, k + 1) @ h.cells[c].lat_inv       # (q, n_lat) Lagrange values
        gf[c] = np.einsum("q,qn,qa->na", wq, lam, uav)
    del npk
    return J, gf, gnu, u, p, ua


def objective(topo, k, fvals, u_target, nu_elem, beta=0.0, gamma=0.0, conv=None):
    h = HDG(topo, k, nu=1.0, beta=beta, gamma=gamma, nu_elem=nu_elem, conv=conv)
    u, p = h.solve_direct(h.load(fvals))
    J = 0.0
    for c in range(topo.n_cells):
        e = _lattice_values(h, c, h.recover_cell(c, u, p[c], fvals[c])) - u_target[c]
        xq, wq = triangle_points(h.cells[c].el.X, k + 4)
        J += 0.5 * wq @ np.sum(_lattice_function(h, c, e, xq) ** 2, axis=1)
    return J
