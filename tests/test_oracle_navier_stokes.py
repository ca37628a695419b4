"""Pins of the oracle's Picard iteration for steady Navier–Stokes (Section 4.2, Algorithm 3 part (i)).

* The fixed point solves the discrete Navier–Stokes problem: re-solving the Oseen
  problem with the converged velocity as convecting field reproduces it.
* Consistency: with f = -νΔu + (u·∇)u + ∇p for the manufactured curl solution the
  converged velocity, flux and pressure converge at order k+1.
* The iteration contracts: successive distances decrease geometrically.
"""
import numpy as np
import pytest

from workloads import curl_bubble_2d, forcing_at_lattice, unit_square
from oracle.hdg import HDG
from oracle.navier_stokes import picard, lattice_velocity, l2_distance
from _util import topo_of

SOL = curl_bubble_2d()


def _ns_forcing(m, k, nu):
    return forcing_at_lattice(m.coords, m.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))


@pytest.mark.parametrize("k", [1, 2])
def test_picard_fixed_point_and_slopes(k):
    nu = 1.0
    errs = []
    for N in (8, 16):
        m = unit_square(N)
        t = topo_of(m)
        fv = _ns_forcing(m, k, nu)
        u, p, n, dist, h, w = picard(t, k, fv, nu, tol=1e-11)
        assert dist < 1e-11 and n < 20
        # fixed point: one more Oseen solve with w = u_h gives u_h back
        h2 = HDG(t, k, nu=nu, conv=w)
        u2, p2 = h2.solve_direct(h2.load(fv))
        assert np.abs(u2 - u).max() < 1e-9 * np.abs(u).max()
        errs.append(h.errors(u, p, fv, SOL))
    for q in ("u", "L", "p"):
        assert np.log2(errs[0][q] / errs[1][q]) > k + 1 - 0.15


def test_picard_contracts():
    m = unit_square(6, shuffle_seed=1)
    t = topo_of(m)
    k, nu = 2, 0.05
    fv = _ns_forcing(m, k, nu)
    h = HDG(t, k, nu=nu)
    u, p = h.solve_direct(h.load(fv))
    prev = lattice_velocity(h, u, p, fv)
    d = []
    for _ in range(5):
        h = HDG(t, k, nu=nu, conv=prev)
        u, p = h.solve_direct(h.load(fv))
        cur = lattice_velocity(h, u, p, fv)
        d.append(l2_distance(h, cur, prev))
        prev = cur
    ratios = [d[i + 1] / d[i] for i in range(4)]
    assert max(ratios) < 0.6


@pytest.mark.parametrize("k,nu", [(1, 0.05), (2, 0.02)])
def test_newton_quadratic_and_same_fixed_point(k, nu):
    """Newton from a rough Picard iterate converges quadratically to the Picard fixed point
    (the same discrete Navier-Stokes solution)."""
    from oracle.navier_stokes import newton
    m = unit_square(6, shuffle_seed=1)
    t = topo_of(m)
    fv = _ns_forcing(m, k, nu)
    up, pp, n, d, h, w = picard(t, k, fv, nu, tol=1e-3)
    un, pn, nn, dists, hn = newton(t, k, fv, nu, h, up, pp, tol=1e-12)
    assert nn <= 4 and dists[-1] < 1e-12
    for a, b in zip(dists, dists[1:]):
        if b > 1e-13:
            assert b < 5.0 * a * a / max(dists[0], 1e-300) + 1e-13 or b < 1e-3 * a
    uP, pP, nP, dP, hP, wP = picard(t, k, fv, nu, tol=1e-13, max_steps=200)
    assert np.abs(un - uP).max() < 1e-11 * np.abs(uP).max()


def test_pseudo_time_picard_same_fixed_point():
    """Pseudo-time continuation (Section 5.2.2) changes the path, not the limit: with
    1/dt* = 0.1 and 1 the Picard iteration converges to the fixed point of the plain one,
    which is the steady discrete solution (re-solving with it as convecting field and
    no pseudo-time term reproduces it)."""
    k, nu = 2, 0.05
    m = unit_square(8)
    t = topo_of(m)
    fv = _ns_forcing(m, k, nu)
    u0, p0, n0, d0, h0, w0 = picard(t, k, fv, nu, gamma=10.0, tol=1e-11)
    for dti in (0.1, 1.0):
        u, p, n, d, h, w = picard(t, k, fv, nu, gamma=10.0, tol=1e-11, pseudo_dt_inv=dti, max_steps=200)
        assert d < 1e-11
        assert np.abs(u - u0).max() < 1e-8 * np.abs(u0).max()
        h2 = HDG(t, k, nu=nu, gamma=10.0, conv=w)
        u2, p2 = h2.solve_direct(h2.load(fv))
        assert np.abs(u2 - u).max() < 1e-8 * np.abs(u).max()
