"""Oracle pins of inhomogeneous Dirichlet data (Section 3.1 with u = g on the boundary;
the driven-lid cavity of Section 5.2).

* Polynomial reproduction: u = (x^2, -2xy) (divergence free), p = x + y - 1 lie in the
  k = 2 spaces, so with their boundary values as data the discrete solution is exact.
* The AL-Uzawa iteration with the data's boundary fluxes reaches the direct solution.
* The driven lid: divergence-free velocity, mean-free pressure, and a data vector with
  zero normal moments (the lid is tangential).
"""
import numpy as np
import pytest

from workloads import unit_square, forcing_at_lattice
from workloads.manufactured import (dirichlet_facet_data, lid_velocity_2d, lattice_barycentric_2d,
                                    boundary_facets_2d)
from oracle.hdg import HDG
from oracle.mg import build_hpmg
from oracle.krylov import uzawa
from _util import hierarchy, topo_of, relnorm

NU, BETA = 0.7, 1.3


def poly_u(x):
    return np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], axis=1)


def poly_f(x):
    return np.stack([-2 * NU + BETA * x[:, 0] ** 2 + 1.0, -2 * BETA * x[:, 0] * x[:, 1] + 1.0], axis=1)


@pytest.mark.parametrize("jitter", [0.0, 0.25])
def test_polynomial_reproduction_with_boundary_data(jitter):
    ms, ts, ps = hierarchy(2, 2, jitter=jitter, seed=4, shuffle_seed=2)
    m, t, k = ms[-1], ts[-1], 2
    data = dirichlet_facet_data(m.coords, m.cells, k, poly_u)
    h = HDG(t, k, nu=NU, beta=BETA, gamma=50.0, dirichlet=data)
    fv = forcing_at_lattice(m.coords, m.cells, k, poly_f)
    u, p = h.solve_direct(h.load(fv))
    lam = lattice_barycentric_2d(k + 1)
    err = 0.0
    for c in range(t.n_cells):
        el = h.cells[c].el
        X0 = t.coords[t.cells[c][0]]
        xl = lam @ el.X
        _, uh, divu, ph = h.fields_at(c, h.recover_cell(c, u, p[c], fv[c]), xl)
        err = max(err, np.abs(uh - poly_u(xl + X0)).max(), np.abs(divu).max())
        err = max(err, np.abs(ph - (xl + X0).sum(axis=1) + 1.0).max())
    assert err < 1e-10
    # the skeleton solution on interior facets equals the data formula evaluated there
    assert h.xD is not None and np.abs(h.boundary_flux()).max() > 0


def test_uzawa_with_boundary_fluxes_reaches_direct_solution():
    ms, ts, ps = hierarchy(2, 3, jitter=0.2, seed=1)
    m, k = ms[-1], 2
    data = dirichlet_facet_data(m.coords, m.cells, k, poly_u)
    h = HDG(ts[-1], k, nu=NU, beta=BETA, gamma=100.0, dirichlet=data)
    M = build_hpmg(ts, ps, k, NU, BETA, 100.0, hdg_k=h)
    F = h.load(forcing_at_lattice(m.coords, m.cells, k, poly_f))
    # the load carries eps^-1 d_I (d_B g) / |K| for data with normal flux: |F| is large, so
    # the floor relative to |F| is set lower than the default
    r = uzawa(M.A, h.flux_matrix(), h.area, h.eps_inv, F, M, bflux=h.boundary_flux(),
              rtol=1e-10, floor_rel=1e-13, uzawa_tol=1e-11)
    u, p = h.solve_direct(F)
    assert relnorm(r.u, u) < 1e-8 and relnorm(r.p, p) < 1e-8
    assert r.div_l2 < 1e-8


def test_driven_lid_cavity():
    ms, ts, ps = hierarchy(2, 3)
    m, k = ms[-1], 2
    data = dirichlet_facet_data(m.coords, m.cells, k, lid_velocity_2d())
    dpf = 2 * (k + 1)
    assert np.abs(data[:, :k + 1]).max() == 0.0          # tangential lid: no normal moments
    pairs = boundary_facets_2d(m.cells)
    top = np.isclose(m.coords[pairs[:, 0], 1], 1.0) & np.isclose(m.coords[pairs[:, 1], 1], 1.0)
    L = np.linalg.norm(m.coords[pairs[:, 1]] - m.coords[pairs[:, 0]], axis=1)
    assert np.allclose(np.abs(data[top, k + 1]), np.sqrt(L[top]))   # |int_F 1 l_0| = sqrt|F|
    assert np.abs(data[~top]).max() == 0.0 and np.abs(data[:, k + 2:dpf]).max() < 1e-14
    h = HDG(ts[-1], k, nu=1.0, beta=0.0, gamma=100.0, dirichlet=data)
    F = h.load(np.zeros((m.n_cells, (k + 2) * (k + 3) // 2, 2)))
    u, p = h.solve_direct(F)
    assert np.abs(h.flux_matrix() @ u + h.boundary_flux()).max() < 1e-12
    assert abs(h.area @ p) < 1e-12
    assert np.linalg.norm(u) > 0.1


def test_backward_facing_step_channel():
    """The backward-facing-step stand-in (non-convex channel, parabolic inflow and outflow of equal
    flux, no-slip walls): the data's boundary fluxes cancel, the AL-Uzawa iteration with the
    hp-multigrid on the red-refined hierarchy reaches the direct solution, and div u_h = 0."""
    from workloads.mesh2d import step_channel_hierarchy
    from workloads.manufactured import step_channel_velocity_2d
    ms = step_channel_hierarchy(3)
    ts = [topo_of(m) for m in ms]
    ps = [m.parent for m in ms]
    m, k = ms[-1], 2
    data = dirichlet_facet_data(m.coords, m.cells, k, step_channel_velocity_2d())
    h = HDG(ts[-1], k, nu=1.0, beta=0.0, gamma=100.0, dirichlet=data)
    bf = h.boundary_flux()
    assert abs(bf.sum()) < 1e-13 and np.abs(bf).max() > 1e-3
    F = h.load(np.zeros((m.n_cells, (k + 2) * (k + 3) // 2, 2)))
    u, p = h.solve_direct(F)
    assert np.abs(h.flux_matrix() @ u + bf).max() < 1e-12
    M = build_hpmg(ts, ps, k, 1.0, 0.0, 100.0, hdg_k=h)
    r = uzawa(M.A, h.flux_matrix(), h.area, h.eps_inv, F, M, bflux=bf, rtol=1e-10, floor_rel=1e-13,
              uzawa_tol=1e-11)
    assert relnorm(r.u, u) < 1e-8 and relnorm(r.p, p) < 1e-8
