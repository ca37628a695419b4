"""GPU parity of the Picard iteration for steady Navier-Stokes (hdg_picard)
against the oracle's Picard iteration with exact solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d, forcing_at_lattice
from oracle.navier_stokes import picard
from _util import hierarchy, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SOL = curl_bubble_2d()


@pytest.mark.parametrize("k,Re,precision", [(1, 1.0, 0), (2, 10.0, 1)])
def test_picard_matches_oracle(k, Re, precision):
    import paper_2303_06762_gb300 as hdg
    nu = 1.0 / Re
    ms, ts, ps = hierarchy(2, 3, shuffle_seed=2)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=100.0, precision=precision)
    u, p, steps, dist = hdg.hdg_picard(ctx, prm, torch.tensor(fv, device=DEV), tol=1e-9, max_steps=40, opts=o)
    uo, po, n, do, h, w = picard(ts[-1], k, fv, nu, gamma=100.0, tol=1e-9)
    assert steps == n
    assert dist < 1e-9
    assert rel(u.cpu().numpy(), uo) < 1e-8
    pm = p.cpu().numpy()
    pm = pm - (h.area @ pm) / h.area.sum()
    pom = po - (h.area @ po) / h.area.sum()
    assert rel(pm, pom) < 1e-7


@pytest.mark.parametrize("dti", [0.1, 1.0])
def test_pseudo_time_picard_matches_oracle(dti):
    """Picard with pseudo-time continuation (Section 5.2.2): the same steps and iterates as the
    oracle's, and the same fixed point as the plain iteration."""
    import paper_2303_06762_gb300 as hdg
    k, nu = 2, 0.05
    ms, ts, ps = hierarchy(2, 3)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=10.0, pseudo_dt_inv=dti)
    u, p, steps, dist = hdg.hdg_picard(ctx, prm, torch.tensor(fv, device=DEV), tol=1e-10, max_steps=200, opts=o)
    uo, po, n, do, h, w = picard(ts[-1], k, fv, nu, gamma=10.0, tol=1e-10, pseudo_dt_inv=dti, max_steps=200)
    u0, *_ = picard(ts[-1], k, fv, nu, gamma=10.0, tol=1e-10)
    print(f"pseudo-time 1/dt*={dti}: {steps} Picard steps (oracle {n})")
    assert abs(steps - n) <= 1
    assert rel(u.cpu().numpy(), uo) < 1e-8 and rel(u.cpu().numpy(), u0) < 1e-8


@pytest.mark.parametrize("k", [1, 2, 3])
def test_newton_operator_matches_oracle(k):
    """Condensed matrices and load of a Newton step (conv = u_old at the lattice, newton_u = the
    previous skeleton iterate) against the oracle's local systems with the Newton term."""
    import paper_2303_06762_gb300 as hdg
    from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
    from oracle.hdg import HDG
    nu, gamma = 0.05, 50.0
    ms, ts, ps = hierarchy(2, 2, shuffle_seed=6)
    fine = ms[-1]
    psi, _ = convecting_stream_2d(1.0)
    w = curl_lattice_2d(fine.coords, fine.cells, k + 1, psi)
    fv = forcing_at_lattice(fine.coords, fine.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))
    oh0 = HDG(ts[-1], k, nu=nu, gamma=gamma)
    x_old = np.random.default_rng(3).standard_normal(oh0.n_dof)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), device=DEV)
    prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=gamma, conv=dv(w), newton_u=dv(x_old))
    F = hdg.hdg_condense(ctx, prm, dv(fv))
    oh = HDG(ts[-1], k, nu=nu, gamma=gamma, conv=w, newton_uhat=oh0.facet_tangential(x_old))
    A = hdg.hdg_get_element_matrices(ctx, -1).cpu().numpy()
    assert rel(A, np.stack([oh.element_matrix(c) for c in range(ts[-1].n_cells)])) < 1e-12
    assert rel(F.cpu().numpy(), oh.load(fv)) < 1e-12


def test_picard_then_newton_matches_oracle():
    """Algorithm 3: Picard to 1e-3, then Newton to 1e-11 (quadratic), against the oracle."""
    import paper_2303_06762_gb300 as hdg
    from oracle.navier_stokes import newton
    k, nu = 2, 0.05
    ms, ts, ps = hierarchy(2, 3, shuffle_seed=2)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=100.0, precision=1)
    f = torch.tensor(fv, device=DEV)
    u, p, n1, d1 = hdg.hdg_picard(ctx, prm, f, tol=1e-3, max_steps=40, opts=o)
    u, p, n2, d2 = hdg.hdg_newton(ctx, prm, f, u, p, tol=1e-11, max_steps=10, opts=o)
    uo, po, m1, e1, h, w = picard(ts[-1], k, fv, nu, gamma=100.0, tol=1e-3)
    uo, po, m2, e2, h2 = newton(ts[-1], k, fv, nu, h, uo, po, gamma=100.0, tol=1e-11)
    assert n1 == m1 and n2 == m2 and n2 <= 4
    assert d2 < 1e-11
    assert rel(u.cpu().numpy(), uo) < 1e-8
