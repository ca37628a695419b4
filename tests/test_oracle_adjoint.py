"""Pin of the oracle's adjoint gradients by central finite differences.

J = 1/2 ||u_h - u_target||^2 with u_h the exact discrete solution (direct
solves); gradients with respect to the forcing lattice values and the
per-cell viscosity (per-cell nu = (1 + 0.1 U[-1,1]), seed 7; directions seed
11, as in the adjoint configuration).  J is quadratic in the forcing and smooth
in nu, so a step of 1e-4 keeps both truncation and cancellation below 1e-7.
"""
import numpy as np
import pytest

from workloads import unit_square, curl_bubble_2d, forcing_at_lattice
from oracle.adjoint import objective_and_gradient, objective
from _util import topo_of


@pytest.mark.parametrize("k,beta", [(1, 0.0), (2, 1.0)])
def test_adjoint_matches_central_differences(k, beta):
    m = unit_square(3, shuffle_seed=2)
    t = topo_of(m)
    rng = np.random.default_rng(7)
    nu = 1.0 * (1 + 0.1 * rng.uniform(-1, 1, t.n_cells))
    fv = forcing_at_lattice(m.coords, m.cells, k, curl_bubble_2d().forcing(1.0, beta))
    ut = forcing_at_lattice(m.coords, m.cells, k, curl_bubble_2d().u) + \
        0.1 * rng.standard_normal(fv.shape)
    J, gf, gn, *_ = objective_and_gradient(t, k, fv, ut, nu, beta=beta)
    assert J > 0
    assert abs(objective(t, k, fv, ut, nu, beta=beta) - J) < 1e-14 * J
    dirs = np.random.default_rng(11)
    h = 1e-4
    for _ in range(10):
        df = dirs.standard_normal(fv.shape)
        dn = 0.1 * dirs.standard_normal(nu.shape)
        fd = (objective(t, k, fv + h * df, ut, nu + h * dn, beta=beta)
              - objective(t, k, fv - h * df, ut, nu - h * dn, beta=beta)) / (2 * h)
        ad = (gf * df).sum() + (gn * dn).sum()
        assert abs(fd - ad) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("k,Re", [(1, 1.0), (2, 100.0)])
def test_oseen_adjoint_matches_central_differences(k, Re):
    """Oseen: the adjoint solve uses the transposed convection block."""
    from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
    psi, b = convecting_stream_2d(1.0)
    m = unit_square(3, shuffle_seed=4)
    t = topo_of(m)
    conv = curl_lattice_2d(m.coords, m.cells, k + 1, psi)
    rng = np.random.default_rng(7)
    nu = (1.0 / Re) * (1 + 0.1 * rng.uniform(-1, 1, t.n_cells))
    fv = forcing_at_lattice(m.coords, m.cells, k, curl_bubble_2d().forcing(1.0 / Re, 0.0, conv=b))
    ut = forcing_at_lattice(m.coords, m.cells, k, curl_bubble_2d().u) + \
        0.1 * rng.standard_normal(fv.shape)
    J, gf, gn, *_ = objective_and_gradient(t, k, fv, ut, nu, conv=conv)
    # the transposed block matters: the Stokes-style adjoint would be wrong here
    J2, gf2, *_ = objective_and_gradient(t, k, fv, ut, nu)
    dirs = np.random.default_rng(11)
    h = 1e-4 / Re
    for _ in range(6):
        df = dirs.standard_normal(fv.shape)
        dn = (0.1 / Re) * dirs.standard_normal(nu.shape)
        fd = (objective(t, k, fv + h * df, ut, nu + h * dn, conv=conv)
              - objective(t, k, fv - h * df, ut, nu - h * dn, conv=conv)) / (2 * h)
        ad = (gf * df).sum() + (gn * dn).sum()
        assert abs(fd - ad) <= 1e-6 * abs(fd)
