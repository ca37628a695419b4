"""Pins of the oracle's Oseen (linearised Navier–Stokes) discretisation, Section 4.

The upwind form of Section 4.1 with a convecting field w_h is pinned by
properties fixed by the mathematics rather than by retyping it:

* consistency: optimal convergence slopes for a manufactured solution whose
  forcing carries the convection term (b·∇)u, so a dropped term, a wrong sign
  or a wrong trace breaks the slopes;
* upwinding: for a divergence-free, normal-continuous w_h with w·n = 0 on ∂Ω
  the convection form equals ½ Σ_K ⟨|w·n|, |tng(u − û)|²⟩ ≥ 0, so the
  symmetric part of its matrix is positive semidefinite (a downwind switch
  or a missing facet term makes it indefinite);
* the condensed matrix of the transposed convection block is the transpose
  of the condensed matrix (a Schur complement identity);
* w = 0 gives back the generalized Stokes matrix exactly;
* the coarse-level fields are divergence free and reproduce constants.
"""
import numpy as np
import pytest

from workloads import curl_bubble_2d, forcing_at_lattice, unit_square
from workloads.manufactured import convecting_stream_2d, curl_lattice_2d, lattice_points_2d
from oracle.hdg import HDG
from oracle.krylov import uzawa
from oracle.mg import build_hpmg, lowest_order_convection

from _util import hierarchy, topo_of

SOL = curl_bubble_2d()
PSI, B = convecting_stream_2d(1.0)


def _conv(mesh, k):
    return curl_lattice_2d(mesh.coords, mesh.cells, k + 1, PSI)


def test_curl_lattice_reproduces_polynomial_streams():
    psi = lambda x: x[:, 0] ** 2 * x[:, 1] - 3 * x[:, 1] ** 2 + x[:, 0]
    m = unit_square(4, shuffle_seed=1)
    w = curl_lattice_2d(m.coords, m.cells, 3, psi).reshape(-1, 2)
    X = lattice_points_2d(m.coords, m.cells, 3).reshape(-1, 2)
    exact = np.stack([X[:, 0] ** 2 - 6 * X[:, 1], -2 * X[:, 0] * X[:, 1] - 1.0], axis=1)
    assert np.abs(w - exact).max() < 1e-12


def test_curl_lattice_converges():
    errs = []
    for N in (8, 16):
        m = unit_square(N, shuffle_seed=3)
        w = curl_lattice_2d(m.coords, m.cells, 3, PSI)
        X = lattice_points_2d(m.coords, m.cells, 3).reshape(-1, 2)
        errs.append(np.abs(w.reshape(-1, 2) - B(X)).max())
    assert np.log2(errs[0] / errs[1]) > 2.7      # degree-3 interpolant: gradient O(h^3)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_upwind_form_is_dissipative(k):
    m = unit_square(5, shuffle_seed=2)
    t = topo_of(m)
    conv = _conv(m, k)
    A = HDG(t, k, nu=0.01, conv=conv).matrix(with_al=False).toarray()
    A0 = HDG(t, k, nu=0.01).matrix(with_al=False).toarray()
    C = A - A0
    scale = np.abs(C).max()
    assert scale > 0.1
    assert np.abs(C - C.T).max() > 0.1 * scale          # genuinely non-symmetric
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > -1e-12 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_transposed_convection_gives_transposed_matrix(k):
    m = unit_square(4, shuffle_seed=5)
    t = topo_of(m)
    conv = _conv(m, k)
    A = HDG(t, k, nu=0.05, beta=1.0, conv=conv).matrix(with_al=False).toarray()
    At = HDG(t, k, nu=0.05, beta=1.0, conv=conv, conv_transpose=True).matrix(with_al=False).toarray()
    assert np.abs(At - A.T).max() < 1e-12 * np.abs(A).max()


def test_zero_field_is_stokes():
    m = unit_square(4, shuffle_seed=5)
    t = topo_of(m)
    conv = np.zeros((m.n_cells, 10, 2))
    A = HDG(t, 2, nu=0.3, beta=2.0, conv=conv).matrix().toarray()
    A0 = HDG(t, 2, nu=0.3, beta=2.0).matrix().toarray()
    assert np.abs(A - A0).max() < 1e-12 * np.abs(A0).max()


@pytest.mark.parametrize("k", [1, 2])
def test_oseen_convergence_slopes(k):
    nu = 1.0
    e = []
    for N in (8, 16):
        m = unit_square(N)
        t = topo_of(m)
        h = HDG(t, k, nu=nu, conv=_conv(m, k))
        fv = forcing_at_lattice(m.coords, m.cells, k, SOL.forcing(nu, 0.0, conv=B))
        u, p = h.solve_direct(h.load(fv))
        e.append(h.errors(u, p, fv, SOL))
    slope = {q: np.log2(e[0][q] / e[1][q]) for q in ("u", "L", "p", "ustar")}
    assert slope["u"] > k + 1 - 0.15
    assert slope["L"] > k + 1 - 0.15
    assert slope["p"] > k + 1 - 0.15
    assert slope["ustar"] > k + 2 - 0.25
    assert e[1]["div"] < 1e-9


def test_lowest_order_fields():
    ms, topos, parents = hierarchy(2, 3, shuffle_seed=4)
    k = 2
    conv = _conv(ms[-1], k)
    fields = lowest_order_convection(topos, parents, conv)
    assert [f.shape for f in fields] == [(t.n_cells, 3, 2) for t in topos]
    for t, w in zip(topos, fields):
        for c in range(t.n_cells):
            X = t.coords[t.cells[c]]
            G = np.linalg.inv(np.stack([X[1] - X[0], X[2] - X[0]], axis=1)).T
            grads = [G @ np.array([-1.0, -1.0]), G @ np.array([1.0, 0.0]), G @ np.array([0.0, 1.0])]
            div = sum(w[c, v] @ grads[v] for v in range(3))
            assert abs(div) < 1e-12
        # normal continuity across interior facets, no flux through the boundary
        for F in range(t.facets.shape[0]):
            lo, hi = t.facets[F]
            xm = 0.5 * (t.coords[lo] + t.coords[hi])
            d = t.coords[hi] - t.coords[lo]
            n = np.array([d[1], -d[0]]) / np.hypot(*d)
            vals = []
            for c in t.facet_cells[F]:
                if c < 0:
                    continue
                X = t.coords[t.cells[c]]
                lam = np.linalg.solve(np.vstack([X.T, np.ones(3)]), np.array([xm[0], xm[1], 1.0]))
                vals.append((lam @ w[c]) @ n)
            if len(vals) == 2:
                assert abs(vals[0] - vals[1]) < 1e-12
            else:
                assert abs(vals[0]) < 1e-12
    const = np.tile(np.array([0.3, -0.7]), (ms[-1].n_cells, conv.shape[1], 1))
    for w in lowest_order_convection(topos, parents, const):
        assert np.abs(w - np.array([0.3, -0.7])).max() < 1e-13


@pytest.mark.parametrize("Re", [1.0, 100.0])
def test_oseen_uzawa_hpmg_reaches_direct_solution(Re):
    ms, topos, parents = hierarchy(2, 3)
    k, nu, gamma = 1, 1.0 / Re, 100.0
    conv = _conv(ms[-1], k)
    mg = build_hpmg(topos, parents, k, nu, 0.0, gamma, conv=conv)
    h = mg.hdg
    fv = forcing_at_lattice(ms[-1].coords, ms[-1].cells, k, SOL.forcing(nu, 0.0, conv=B))
    F = h.load(fv)
    ud, pd = h.solve_direct(F)
    res = uzawa(h.matrix(with_al=True), h.flux_matrix(), h.area, h.eps_inv, F, mg,
                rtol=1e-10, atol=1e-13, restart=30, max_it=400, max_uzawa=60, uzawa_tol=1e-10)
    assert np.abs(res.u - ud).max() < 1e-7 * np.abs(ud).max()
    pm = res.p - (h.area @ res.p) / h.area.sum()
    pdm = pd - (h.area @ pd) / h.area.sum()
    assert np.abs(pm - pdm).max() < 1e-6 * np.abs(pdm).max()
    assert max(res.krylov_its) < 40
