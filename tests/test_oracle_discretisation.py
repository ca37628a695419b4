"""Pins of the oracle's discretisation against facts the paper or mathematics fix.

* quadrature: exact monomial integrals on the reference triangle;
* spaces: unisolvence of the RT_k degrees of freedom, orthonormal facet basis;
* condensation: the condensed solve + recovery equals the brute-force
  solve of the uncondensed global system (Section 3.2);
* convergence orders k+1 for u_h and L_h, k+2 for u* (Section 5.1);
* exact divergence-free velocity (div V_h^k = W_h^k, Section 3.2);
* pressure robustness (Section 1, Section 3.2): a gradient added to f only
  changes p_h, by the L2 projection of the potential;
* A^ε symmetric positive definite (Section 3.2);
* independence of the skeleton operator from the cells' local vertex order.
"""
from math import factorial

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import unit_square, curl_bubble_2d, polynomial_2d, forcing_at_lattice
from workloads.manufactured import gradient_field_2d
from oracle.quadrature import gauss_legendre_01, triangle_rule, triangle_points
from oracle.spaces import Element, exponents
from oracle.hdg import HDG, local_system
from _util import topo_of, forcing, rel


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_triangle_rule_exact(n):
    pts, w = triangle_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(w @ (pts[:, 0] ** a * pts[:, 1] ** b) - exact) < 1e-15
    s, w1 = gauss_legendre_01(n)
    for a in range(2 * n):
        assert abs(w1 @ s ** a - 1 / (a + 1)) < 1e-15


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_rt_unisolvence_and_facet_basis(k):
    X = np.array([[0.1, 0.2], [0.9, 0.35], [0.3, 1.1]])
    el = Element(X, [7, 2, 5], k)
    assert el.n_rt == (k + 1) * (k + 3)
    # facet moments of the facet basis functions are the identity
    for f in range(3):
        s, xf, wf = el.facet_points(f, k + 3)
        U = el.rt_values(xf) @ el.facets[f]["nF"]          # (q, n_rt)
        lm = el.facet_legendre(f, s)
        mom = (lm * wf[:, None]).T @ U                     # (k+1, n_rt)
        expect = np.zeros_like(mom)
        for m in range(k + 1):
            expect[m, f * (k + 1) + m] = 1.0
        assert np.abs(mom - expect).max() < 1e-10
        assert np.abs((lm * wf[:, None]).T @ lm - np.eye(k + 1)).max() < 1e-13
    # divergence of RT_k lies in P^k: exact fit by monomials of degree k
    xq, wq = triangle_points(X, k + 3)
    D = el.rt_div(xq)
    P = el.mono(xq, k)
    coef, *_ = np.linalg.lstsq(P, D, rcond=None)
    assert np.abs(P @ coef - D).max() < 1e-10 * max(1, np.abs(D).max())


def _brute_force_solve(topo, k, nu, beta, fv):
    """Uncondensed global system: all unknowns (L, u, û, p) assembled, dense solve."""
    nc = topo.n_cells
    npk = len(exponents(k))
    nL = 4 * npk
    n_int_rt = k * (k + 1)
    nf = topo.facets.shape[0]
    # global numbering: facet normal moments, facet tangential, cell locals
    off_un = 0
    off_uh = nf * (k + 1)
    off_cell = 2 * nf * (k + 1)
    per_cell = nL + n_int_rt + npk
    n = off_cell + nc * per_cell + 1          # + mean-zero multiplier
    K = np.zeros((n, n))
    R = np.zeros(n)
    for c in range(nc):
        gv = topo.cells[c]
        el = Element(topo.coords[gv], gv, k)
        M, rhs_map, g, loc, p0, _, o = local_system(el, nu, beta)
        rhs = rhs_map @ fv[c].reshape(-1)
        idx = np.empty(M.shape[0], dtype=np.int64)
        base = off_cell + c * per_cell
        idx[o["oL"]:o["oL"] + nL] = base + np.arange(nL)
        for f in range(3):
            F = topo.cell_facets[c, f]
            idx[o["ou"] + f * (k + 1):o["ou"] + (f + 1) * (k + 1)] = off_un + F * (k + 1) + np.arange(k + 1)
            idx[o["oh"] + f * (k + 1):o["oh"] + (f + 1) * (k + 1)] = off_uh + F * (k + 1) + np.arange(k + 1)
        idx[o["ou"] + 3 * (k + 1):o["ou"] + o["nrt"]] = base + nL + np.arange(n_int_rt)
        idx[o["op"]:o["op"] + npk] = base + nL + n_int_rt + np.arange(npk)
        K[np.ix_(idx, idx)] += M
        R[idx] += rhs
        # mean-zero pressure: only the constant mode has nonzero mean
        K[n - 1, base + nL + n_int_rt] = el.area
        K[base + nL + n_int_rt, n - 1] = el.area
    bnd = [F for F in range(nf) if topo.facet_cells[F, 1] < 0]
    fix = []
    for F in bnd:
        fix += list(off_un + F * (k + 1) + np.arange(k + 1)) + list(off_uh + F * (k + 1) + np.arange(k + 1))
    keep = np.setdiff1d(np.arange(n), fix)
    sol = np.zeros(n)
    sol[keep] = np.linalg.solve(K[np.ix_(keep, keep)], R[keep])
    return sol, off_un, off_uh, off_cell, per_cell


@pytest.mark.parametrize("k", [0, 1, 2])
def test_condensation_equals_brute_force(k):
    m = unit_square(2, shuffle_seed=3)
    topo = topo_of(m)
    sol = curl_bubble_2d()
    nu, beta = 0.7, 2.0
    fv = forcing(m, k, sol, nu, beta)
    h = HDG(topo, k, nu=nu, beta=beta, cache=False)
    u, p = h.solve_direct(h.load(fv))
    bf, off_un, off_uh, off_cell, per_cell = _brute_force_solve(topo, k, nu, beta, fv)
    dpf = 2 * (k + 1)
    for i, F in enumerate(topo.interior_facets):
        assert np.allclose(u[i * dpf:i * dpf + k + 1], bf[off_un + F * (k + 1):off_un + (F + 1) * (k + 1)],
                           atol=1e-11)
        assert np.allclose(u[i * dpf + k + 1:(i + 1) * dpf], bf[off_uh + F * (k + 1):off_uh + (F + 1) * (k + 1)],
                           atol=1e-11)
    npk = len(exponents(k))
    for c in range(topo.n_cells):
        Lc, rt, pc = h.recover_cell(c, u, p[c], fv[c])
        base = off_cell + c * per_cell
        assert np.allclose(Lc.ravel(), bf[base:base + 4 * npk], atol=1e-10)
        assert np.allclose(pc, bf[base + 4 * npk + k * (k + 1):base + per_cell], atol=1e-10)


def _eoc_run(k, sol, Ns, nu=1.0, beta=1.0):
    errs = []
    for N in Ns:
        m = unit_square(N)
        h = HDG(topo_of(m), k, nu=nu, beta=beta)
        fv = forcing(m, k, sol, nu, beta)
        u, p = h.solve_direct(h.load(fv))
        errs.append(h.errors(u, p, fv, sol))
    return errs


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_convergence_orders(k):
    errs = _eoc_run(k, curl_bubble_2d(), [8, 16])
    for key, order in (("u", k + 1), ("L", k + 1)):
        eoc = np.log2(errs[0][key] / errs[1][key])
        assert abs(eoc - order) < 0.2, (key, eoc)
    if k >= 1:
        eoc = np.log2(errs[0]["ustar"] / errs[1]["ustar"])
        assert abs(eoc - (k + 2)) < 0.2, ("ustar", eoc)
    # ‖∇u‖_{L2} of the curl bubble is about 6; the divergence is round-off
    for e in errs:
        assert e["div"] < 1e-8


def test_convergence_polynomial_solution():
    """The paper's own 2D solution (Section 5.1)."""
    errs = _eoc_run(2, polynomial_2d(), [4, 8, 16], beta=0.0)
    eocs = [np.log2(errs[i]["u"] / errs[i + 1]["u"]) for i in range(2)]
    assert abs(eocs[-1] - 3) < 0.2
    assert abs(np.log2(errs[1]["ustar"] / errs[2]["ustar"]) - 4) < 0.25


@pytest.mark.parametrize("k", [1, 2])
def test_pressure_robustness(k):
    m = unit_square(4, shuffle_seed=1)
    topo = topo_of(m)
    sol = curl_bubble_2d()
    h = HDG(topo, k, nu=1.0, beta=1.0)
    fv = forcing(m, k, sol, 1.0, 1.0)
    a = np.random.default_rng(5).standard_normal((k + 2, k + 2))
    phi, gphi = gradient_field_2d(a)
    fv2 = fv + forcing_at_lattice(m.coords, m.cells, k, gphi)
    u1, p1 = h.solve_direct(h.load(fv))
    u2, p2 = h.solve_direct(h.load(fv2))
    assert np.abs(u2 - u1).max() < 1e-10 * np.abs(u1).max()
    # p changes by the L2 projection of phi onto W_h^k (minus its mean)
    diffs, projs, ws = [], [], []
    for c in range(topo.n_cells):
        el = h.cells[c].el
        X0 = topo.coords[topo.cells[c][0]]
        xq, wq = triangle_points(el.X, k + 4)
        _, _, _, pa = h.fields_at(c, h.recover_cell(c, u1, p1[c], fv[c]), xq)
        _, _, _, pb = h.fields_at(c, h.recover_cell(c, u2, p2[c], fv2[c]), xq)
        P = el.mono(xq, k)
        Mp = (P * wq[:, None]).T @ P
        coef = np.linalg.solve(Mp, (P * wq[:, None]).T @ phi(xq + X0))
        diffs.append(pb - pa)
        projs.append(P @ coef)
        ws.append(wq)
    d, pr, w = map(np.concatenate, (diffs, projs, ws))
    pr = pr - (w @ pr) / w.sum()
    assert np.abs(d - pr).max() < 1e-9 * np.abs(pr).max()


@pytest.mark.parametrize("k", [0, 2])
def test_operator_spd_and_orientation_independent(k):
    m1 = unit_square(3)
    m2 = unit_square(3, shuffle_seed=11)
    A1 = HDG(topo_of(m1), k, nu=1.3, beta=0.5, gamma=100.0).matrix().toarray()
    A2 = HDG(topo_of(m2), k, nu=1.3, beta=0.5, gamma=100.0).matrix().toarray()
    assert np.abs(A1 - A1.T).max() < 1e-12 * np.abs(A1).max()
    assert np.linalg.eigvalsh(0.5 * (A1 + A1.T)).min() > 0
    assert rel(A2, A1) < 1e-12
