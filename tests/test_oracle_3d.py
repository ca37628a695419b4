"""Pins of the 3D oracle (tetrahedra; Section 2 with d = 3, Section 3.4.2 edge patches,
Section 5.1.2 workloads).

* Meshes: the Kuhn tetrahedrisation's counts (6n³ cells, 12n³ + 6n² faces, 12n² of them
  on the boundary) and Bey's red refinement, which maps unit_cube(n) onto unit_cube(2n)
  cell for cell with the vertex order kept.
* Quadrature: the conical product rule integrates x^a y^b z^c exactly.
* RT_k: the face basis is orthonormal; the dual basis reproduces [P^k]³ and x P~^k
  fields from their degrees of freedom; each face function has zero normal trace on
  the other faces and interior functions on all faces.
* Polynomial reproduction: u = (x² + yz, −2xy + xz, xy) (divergence free) and
  p = x + y + z − 3/2 lie in the k = 2 spaces, so with their boundary data the discrete
  solution is exact on jittered, reoriented meshes (every term of eq. stWeak enters).
* Theorem 3.1 in 3D: the condensed k = 0 operator and load equal an independently
  assembled Crouzeix–Raviart system (with Π^RT in the β and load terms) under Π^CR.
* Convergence: order k+1 for u_h (manufactured curl solution of the 3D configs).
* Pressure robustness: a gradient added to f leaves u_h unchanged.
* hp-multigrid on edge patches: proper colouring, patch coverage, symmetric MG_hp, and
  the AL-Uzawa iteration reaches the exact discrete solution.
"""
from math import factorial

import numpy as np
import pytest

from workloads.manufactured import curl_bubble_3d, forcing_at_lattice
from workloads.mesh3d import unit_cube, unit_cube_hierarchy, boundary_faces_3d
from oracle.quadrature import tetrahedron_rule, tetrahedron_points
from oracle.topology3d import build_topology_3d, edge_patches
from oracle.spaces3d import Element3, exponents3, homogeneous_exponents3
from oracle.hdg3d import HDG3D, dirichlet_data_3d
from oracle.cr3d import cr_system_3d, pi_cr_matrix_3d
from oracle.mg3d import build_hpmg_3d
from oracle.krylov import uzawa
from _util import rel, relnorm

NU, BETA = 0.7, 1.3


def topo3(m):
    return build_topology_3d(m.coords, m.cells)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_kuhn_counts_and_bey_refinement(n):
    m = unit_cube(n)
    t = topo3(m)
    assert m.n_cells == 6 * n ** 3
    assert t.facets.shape[0] == 12 * n ** 3 + 6 * n ** 2
    assert len(boundary_faces_3d(m.cells)) == 12 * n ** 2 == t.facets.shape[0] - t.n_interior
    vol = np.array([t.cell_volume(c) for c in range(t.n_cells)])
    assert abs(vol.sum() - 1.0) < 1e-13 and np.allclose(vol, 1.0 / (6 * n ** 3))
    fine = unit_cube_hierarchy(n, 2)[-1]
    ref = unit_cube(2 * n)

    def cells_as_points(mm):
        return {tuple(map(tuple, np.round(mm.coords[c] * 2 * n).astype(int))) for c in mm.cells}
    assert cells_as_points(fine) == cells_as_points(ref)
    assert np.all(fine.parent == np.repeat(np.arange(m.n_cells), 8))


def test_tetrahedron_rule_exact():
    for n in range(1, 5):
        p, w = tetrahedron_rule(n)
        for a in range(2 * n):
            for b in range(2 * n - a):
                for c in range(2 * n - a - b):
                    exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                    assert abs(w @ (p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c) - exact) < 1e-15


@pytest.mark.parametrize("k", [0, 1, 2])
def test_rt3_basis(k):
    rng = np.random.default_rng(k)
    X = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.1]]) + rng.uniform(-0.1, 0.1, (4, 3))
    el = Element3(X, [7, 2, 9, 4], k)
    nf = el.nf
    assert el.n_rt == (k + 1) * (k + 2) * (k + 4) // 2
    # orthonormal face bases
    for f in range(4):
        _, lm, w = el.face_quad(f, k + 3)
        assert np.abs((lm * w[:, None]).T @ lm - np.eye(nf)).max() < 1e-12
    # degrees of freedom of a field (face moments, interior moments) -> the dual basis
    def dofs(fun):
        out = []
        for f in range(4):
            x, lm, w = el.face_quad(f, k + 4)
            out += list((w * (fun(x) @ el.facets[f]["nF"])) @ lm)
        if k >= 1:
            xq, wq = tetrahedron_points(el.X, k + 3)
            P = el.mono(xq, k - 1)
            v = fun(xq)
            out += [(wq * P[:, r]) @ v[:, a] for a in range(3) for r in range(P.shape[1])]
        return np.array(out)
    xt, _ = tetrahedron_points(el.X, 3)
    for trial in range(3):
        cP = rng.standard_normal((len(exponents3(k)), 3))
        ch = rng.standard_normal(len(homogeneous_exponents3(k)))
        H = [exponents3(k).index(e) for e in homogeneous_exponents3(k)]

        def fun(x):
            M = el.mono(x, k)
            return M @ cP + el.xi(x) * (M[:, H] @ ch)[:, None]
        assert np.abs(np.einsum("qic,i->qc", el.rt_values(xt), dofs(fun)) - fun(xt)).max() < 1e-11
    # normal traces: face-f functions vanish on the other faces, interior ones on all faces
    for g in range(4):
        x, _, _ = el.face_quad(g, 3)
        vn = el.rt_values(x) @ el.facets[g]["nF"]
        others = [i for i in range(el.n_rt) if not (g * nf <= i < (g + 1) * nf)]
        assert np.abs(vn[:, others]).max() < 1e-11


def _poly(x):
    return np.stack([x[:, 0] ** 2 + x[:, 1] * x[:, 2], -2 * x[:, 0] * x[:, 1] + x[:, 0] * x[:, 2],
                     x[:, 0] * x[:, 1]], axis=1)


def _poly_forcing(x):
    u = _poly(x)
    return np.stack([-2 * NU + BETA * u[:, 0] + 1, BETA * u[:, 1] + 1, BETA * u[:, 2] + 1], axis=1)


class _PolySolution:
    u = staticmethod(_poly)

    @staticmethod
    def grad_u(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return np.stack([np.stack([2 * X, Z, Y], 1), np.stack([-2 * Y + Z, -2 * X, X], 1),
                         np.stack([Y, X, 0 * X], 1)], axis=1)

    @staticmethod
    def p(x):
        return x.sum(axis=1) - 1.5


@pytest.mark.parametrize("jitter", [0.0, 0.25])
def test_polynomial_reproduction(jitter):
    m = unit_cube_hierarchy(2, 1, jitter=jitter, seed=3, shuffle_seed=1 if jitter else None)[-1]
    t = topo3(m)
    k = 2
    h = HDG3D(t, k, nu=NU, beta=BETA, gamma=50.0, dirichlet=dirichlet_data_3d(t, k, _poly))
    fv = forcing_at_lattice(m.coords, m.cells, k, _poly_forcing)
    u, p = h.solve_direct(h.load(fv))
    e = h.errors(u, p, fv, _PolySolution)
    assert e["u"] < 1e-11 and e["L"] < 1e-10 and e["p"] < 1e-10 and e["div"] < 1e-10


@pytest.mark.parametrize("beta", [0.0, 3.0])
def test_theorem_3_1_in_3d(beta):
    m = unit_cube_hierarchy(2, 1, jitter=0.3, seed=7, shuffle_seed=2)[-1]
    t = topo3(m)
    nu, gamma = 1.7, 50.0
    h = HDG3D(t, 0, nu=nu, beta=beta, gamma=gamma)
    fv = forcing_at_lattice(m.coords, m.cells, 0, curl_bubble_3d().forcing(nu, beta))
    Acr, Fcr = cr_system_3d(t, nu, beta, gamma * nu, fv)
    T = pi_cr_matrix_3d(t)
    assert rel((T.T @ Acr @ T).toarray(), h.matrix().toarray()) < 1e-13
    assert rel(T.T @ Fcr, h.load(fv)) < 1e-13


def test_convergence_order_k1():
    """k = 1, n = 4 -> 8 (51,840 unknowns, exact AL-Uzawa solve): order 2 for u_h, L_h, p_h."""
    sol = curl_bubble_3d()
    errs = []
    for nl in (2, 3):
        m = unit_cube_hierarchy(2, nl)[-1]
        h = HDG3D(topo3(m), 1, nu=1.0, beta=1.0, gamma=100.0)
        fv = forcing_at_lattice(m.coords, m.cells, 1, sol.forcing(1.0, 1.0))
        u, p = h.solve_al_exact(h.load(fv))
        errs.append(h.errors(u, p, fv, sol))
    for key in ("u", "L", "p"):
        assert abs(np.log2(errs[0][key] / errs[1][key]) - 2.0) < 0.15, key
    assert errs[1]["div"] < 1e-9


def test_exact_al_solve_matches_saddle_point_solve():
    m = unit_cube_hierarchy(2, 2)[-1]
    h = HDG3D(topo3(m), 1, nu=1.0, beta=1.0, gamma=100.0)
    F = h.load(forcing_at_lattice(m.coords, m.cells, 1, curl_bubble_3d().forcing(1.0, 1.0)))
    u1, p1 = h.solve_direct(F)
    u2, p2 = h.solve_al_exact(F)
    assert relnorm(u2, u1) < 1e-11 and relnorm(p2, p1) < 1e-8


def test_pressure_robustness():
    m = unit_cube_hierarchy(2, 1, shuffle_seed=5)[-1]
    t = topo3(m)
    k = 1
    h = HDG3D(t, k, nu=1.0, beta=1.0, gamma=10.0)
    sol = curl_bubble_3d()
    fv = forcing_at_lattice(m.coords, m.cells, k, sol.forcing(1.0, 1.0))
    a = np.random.default_rng(5).standard_normal(4)

    def gphi(x):     # grad of phi = a0 x² y + a1 y z² + a2 x y z + a3 z³ (degree 3 = k + 2)
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return np.stack([2 * a[0] * X * Y + a[2] * Y * Z, a[0] * X ** 2 + a[1] * Z ** 2 + a[2] * X * Z,
                         2 * a[1] * Y * Z + a[2] * X * Y + 3 * a[3] * Z ** 2], axis=1)
    u1, _ = h.solve_direct(h.load(fv))
    u2, _ = h.solve_direct(h.load(fv + forcing_at_lattice(m.coords, m.cells, k, gphi)))
    assert np.abs(u2 - u1).max() < 1e-10 * np.abs(u1).max()


def test_edge_patches_colouring_and_coverage():
    m = unit_cube_hierarchy(2, 2, jitter=0.2, seed=2)[-1]
    t = topo3(m)
    for c in range(t.n_cells):
        cols = t.edge_colour[t.cell_edges[c]]
        assert len(set(cols.tolist())) == 6            # the six edges of a cell differ
    pts = edge_patches(t, 3)
    count = np.zeros(3 * t.n_interior, dtype=int)
    for _, d in pts:
        count[d] += 1
    assert np.all(count == 3)                           # a face lies in the patches of its 3 edges
    assert max(len(d) for _, d in pts) // 3 <= 8


@pytest.mark.parametrize("k", [1, 2])
def test_hpmg_symmetric_and_uzawa_reaches_discrete_solution(k):
    ms = unit_cube_hierarchy(1, 3)
    ts = [topo3(m) for m in ms]
    ps = [m.parent for m in ms]
    h = HDG3D(ts[-1], k, nu=1.0, beta=1.0, gamma=100.0)
    M = build_hpmg_3d(ts, ps, k, 1.0, 1.0, 100.0, hdg_k=h)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(h.n_dof), rng.standard_normal(h.n_dof)
    assert abs(y @ M(x) - x @ M(y)) < 1e-10 * abs(y @ M(x))
    assert x @ M(x) > 0
    F = h.load(forcing_at_lattice(ms[-1].coords, ms[-1].cells, k, curl_bubble_3d().forcing(1.0, 1.0)))
    r = uzawa(M.A, h.flux_matrix(), h.area, h.eps_inv, F, M, rtol=1e-10, floor_rel=1e-13, uzawa_tol=1e-11)
    u, p = h.solve_al_exact(F)
    assert relnorm(r.u, u) < 1e-8 and relnorm(r.p, p) < 1e-7
    assert max(r.krylov_its) <= 60          # rtol 1e-10 (the default 1e-8 takes 33 at k = 2)


def test_two_level_robust_in_h_and_gamma():
    """The lowest-order two-level method on tetrahedra (edge-patch block GS with m = 2, the averaging
    transfer with harmonic extension, exact coarse solve) as a PCG preconditioner: the counts for a
    random load stay flat from n = 4 to 8 and do not depend on gamma (Theorem 3.2's robustness,
    checked in 3D; measured 14, 17 and 17 at n = 16)."""
    from oracle.krylov import pcg
    counts = {}
    for nc in (2, 4):
        ms = unit_cube_hierarchy(nc, 2)
        ts = [topo3(m) for m in ms]
        ps = [m.parent for m in ms]
        b = None
        for gamma in (1e2, 1e4):
            h = HDG3D(ts[-1], 0, nu=1.0, beta=0.0, gamma=gamma)
            M = build_hpmg_3d(ts, ps, 0, 1.0, 0.0, gamma, m_p=2, m_h=2, hdg_k=h)
            b = np.random.default_rng(0).standard_normal(h.n_dof) if b is None else b
            counts[(nc, gamma)] = pcg(M.A, b, np.zeros_like(b), M)[1]
    vals = list(counts.values())
    assert max(vals) <= 18 and max(vals) - min(vals) <= 4, counts
    assert abs(counts[(4, 1e2)] - counts[(4, 1e4)]) <= 1 and abs(counts[(2, 1e2)] - counts[(2, 1e4)]) <= 1


def test_postprocessing_reproduces_quadratic_velocity():
    """u* of eq. stPost on tetrahedra: with the quadratic divergence-free solution and its boundary
    data at k = 2 (u_h and L_h exact), u* equals u at every lattice point; with a sign or scale error
    in the gradient equation or the mean closure it would not."""
    from workloads.manufactured import lattice_barycentric_3d
    m = unit_cube_hierarchy(2, 1, jitter=0.2, seed=5, shuffle_seed=3)[-1]
    t = topo3(m)
    k = 2
    h = HDG3D(t, k, nu=NU, beta=BETA, gamma=50.0, dirichlet=dirichlet_data_3d(t, k, _poly))
    fv = forcing_at_lattice(m.coords, m.cells, k, _poly_forcing)
    u, p = h.solve_direct(h.load(fv))
    us = h.postprocess(u, p, fv)
    xl = np.einsum("pv,cvd->cpd", lattice_barycentric_3d(k + 1), m.coords[m.cells])
    assert np.abs(us - _poly(xl.reshape(-1, 3)).reshape(xl.shape)).max() < 1e-9
