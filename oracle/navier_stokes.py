"""Picard and Newton iterations for the steady Navier–Stokes equations (oracle).

TEST INFRASTRUCTURE ONLY.

Section 4.2, Algorithm 3 part (i): u^(0) solves the generalized Stokes problem
with the same data; step n solves the Oseen problem of eq. nsWeak (Picard form,
f' = f) whose convecting field is the previous velocity, w_h = u_h^(n-1), and
the iteration stops when ||u_h^(n) - u_h^(n-1)||_{L2(Ω)} < tol.  The velocity
u_h ∈ RT_k ⊂ [P^{k+1}]² is handed to the next step as its values at each cell's
degree-(k+1) lattice (exact), the layout of the convecting field.  Every solve
is a sparse direct solve of the condensed saddle point.

Part (ii), Newton: with the previous iterate (u_old, û_old), solve the scheme
with C_h(u_old; u, v) + C_h(u; u_old, v) in place of the convection term and
C_h(u_old; u_old, v) added to the load: the Newton step of eq. nsWeak written for
the new iterate u = u_old + δu (the switch of the upwind trace frozen at
u_old·n_K), until ||u^(n) - u^(n-1)||_{L2} < tol.
"""

from __future__ import annotations

import numpy as np

from workloads.manufactured import lattice_barycentric_2d

from .hdg import HDG
from .quadrature import triangle_points


def lattice_velocity(h: HDG, u: np.ndarray, p: np.ndarray, fvals: np.ndarray) -> np.ndarray:
    """(n_cells, n_lat(k+1), 2) values of u_h at every cell's degree-(k+1) lattice."""
    out = []
    for c in range(h.topo.n_cells):
        el = h.cells[c].el
        Xl = lattice_barycentric_2d(h.k + 1) @ el.X
        _, uv, _, _ = h.fields_at(c, h.recover_cell(c, u, p[c], fvals[c]), Xl)
        out.append(uv)
    return np.stack(out)


def l2_distance(h: HDG, a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_{L2(Ω)} for two lattice-valued [P^{k+1}]² fields."""
    s = 0.0
    for c in range(h.topo.n_cells):
        cc = h.cells[c]
        xq, wq = triangle_points(cc.el.X, h.k + 4)
        v = cc.el.mono(xq, h.k + 1) @ (cc.lat_inv @ (a[c] - b[c]))
        s += wq @ np.sum(v ** 2, axis=1)
    return float(np.sqrt(s))


def picard(topo, k, fvals, nu, beta=0.0, gamma=0.0, tol=1e-8, max_steps=50, pseudo_dt_inv=0.0):
    """Returns (u, p, steps, last distance, the HDG object of the last step, lattice velocity).

    pseudo_dt_inv = 1/δt* > 0 adds the pseudo-time continuation of Section 5.2.2 to the Oseen
    steps: the backward-Euler step (u^n − u^{n−1})/δt* + (Oseen operator)u^n = f, i.e. β + 1/δt*
    and the load f + u^{n−1}/δt* (u^{n−1} ∈ RT_k ⊂ [P^{k+1}]² given exactly by its lattice
    values); a fixed point of the iteration is the steady solution."""
    h = HDG(topo, k, nu=nu, beta=beta, gamma=gamma)
    u, p = h.solve_direct(h.load(fvals))
    prev = lattice_velocity(h, u, p, fvals)
    dist = np.inf
    n = 0
    for n in range(1, max_steps + 1):
        h = HDG(topo, k, nu=nu, beta=beta + pseudo_dt_inv, gamma=gamma, conv=prev)
        fn = fvals + pseudo_dt_inv * prev
        u, p = h.solve_direct(h.load(fn))
        cur = lattice_velocity(h, u, p, fn)
        dist = l2_distance(h, cur, prev)
        prev = cur
        if dist < tol:
            break
    return u, p, n, dist, h, prev


def newton(topo, k, fvals, nu, h_start, u_start, p_start, beta=0.0, gamma=0.0, tol=1e-10, max_steps=20):
    """Newton iteration from the skeleton iterate (u_start, p_start) computed with the
    HDG object h_start (e.g. the last Picard step, whose local systems recover it).
    Returns (u, p, steps, distances per step, HDG of the last step)."""
    u, p, hp = u_start, p_start, h_start
    dists = []
    for _ in range(max_steps):
        w = lattice_velocity(hp, u, p, fvals)
        uh = hp.facet_tangential(u)
        h_new = HDG(topo, k, nu=nu, beta=beta, gamma=gamma, conv=w, newton_uhat=uh)
        un, pn = h_new.solve_direct(h_new.load(fvals))
        wn = lattice_velocity(h_new, un, pn, fvals)
        dists.append(l2_distance(h_new, wn, w))
        u, p, hp = un, pn, h_new
        if dists[-1] < tol:
            break
    return u, p, len(dists), dists, hp
