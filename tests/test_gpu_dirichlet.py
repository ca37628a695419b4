"""GPU parity with inhomogeneous Dirichlet data (hdg_params.dirichlet): polynomial
reproduction, the driven-lid cavity of Section 5.2 (structured stand-in mesh) against the
oracle, its PCG counts beside the paper's, and the unsupported combinations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import forcing_at_lattice
from workloads.manufactured import dirichlet_facet_data, lid_velocity_2d, lattice_barycentric_2d
from oracle.hdg import HDG
from oracle.mg import build_hpmg
from oracle.krylov import uzawa
from _util import hierarchy, rel, relnorm, parity_opts

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NU, BETA = 0.7, 1.3


def poly_u(x):
    return np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], axis=1)


def poly_f(x):
    return np.stack([-2 * NU + BETA * x[:, 0] ** 2 + 1.0, -2 * BETA * x[:, 0] * x[:, 1] + 1.0], axis=1)


def test_boundary_facet_order_and_polynomial_reproduction():
    import paper_2303_06762_gb300 as hdg
    from workloads.manufactured import boundary_facets_2d
    k = 2
    ms, ts, ps = hierarchy(2, 3, jitter=0.2, seed=6, shuffle_seed=3)
    m = ms[-1]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    assert np.array_equal(hdg.hdg_boundary_facets(ctx), boundary_facets_2d(m.cells))
    data = dirichlet_facet_data(m.coords, m.cells, k, poly_u)
    fv = forcing_at_lattice(m.coords, m.cells, k, poly_f)
    prm = hdg.Params(k=k, nu=NU, beta=BETA, gamma=100.0, dirichlet=torch.tensor(data, device=DEV))
    F = hdg.hdg_condense(ctx, prm, torch.tensor(fv, device=DEV))
    oh = HDG(ts[-1], k, nu=NU, beta=BETA, gamma=100.0, dirichlet=data)
    assert rel(F.cpu().numpy(), oh.load(fv)) < 1e-12
    o = parity_opts(hdg, 100.0)
    o.floor_rel = 1e-13          # |F| carries the AL coupling of the data's normal fluxes
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    _, ul = hdg.hdg_recover(ctx, u, torch.tensor(fv, device=DEV))
    lam = lattice_barycentric_2d(k + 1)
    xl = np.einsum("pv,cvd->cpd", lam, m.coords[m.cells])
    assert np.abs(ul.cpu().numpy() - poly_u(xl.reshape(-1, 2)).reshape(xl.shape)).max() < 1e-9
    assert info["div_l2"] < 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_driven_lid_matches_oracle(precision):
    import paper_2303_06762_gb300 as hdg
    k, gamma = 2, 1e4
    ms, ts, ps = hierarchy(2, 4)
    m = ms[-1]
    data = dirichlet_facet_data(m.coords, m.cells, k, lid_velocity_2d())
    zero = np.zeros((m.n_cells, (k + 2) * (k + 3) // 2, 2))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=1.0, beta=0.0, gamma=gamma, precision=precision,
                     dirichlet=torch.tensor(data, device=DEV))
    F = hdg.hdg_condense(ctx, prm, torch.tensor(zero, device=DEV))
    oh = HDG(ts[-1], k, nu=1.0, beta=0.0, gamma=gamma, dirichlet=data)
    Fo = oh.load(zero)
    assert rel(F.cpu().numpy(), Fo) < 1e-12
    ud, pd = oh.solve_direct(Fo)
    u, p, info = hdg.hdg_solve(ctx, F)
    eu, ep = relnorm(u.cpu().numpy(), ud), relnorm(p.cpu().numpy(), pd)
    print(f"lid, precision {precision}: its {info['krylov_its']} vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-8 and ep < 1e-8
    if precision == 0:
        M = build_hpmg(ts, ps, k, 1.0, 0.0, gamma, hdg_k=oh)
        ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, Fo, M, bflux=oh.boundary_flux(), krylov="pcg")
        o = hdg.default_solve_opts()
        o.krylov = 1
        u, p, info = hdg.hdg_solve(ctx, F, opts=o)
        assert info["krylov_its"] == ro.krylov_its
        assert relnorm(u.cpu().numpy(), ro.u) < 1e-10
    # u* with the lid data on the boundary matches the oracle's
    us = hdg.hdg_postprocess(ctx, torch.tensor(ud, device=DEV), torch.tensor(zero, device=DEV))
    assert rel(us.cpu().numpy(), oh.postprocess(ud, pd, zero)) < 1e-10
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_solve_multi(ctx, F[None].contiguous())
    assert e.value.status == 8


@pytest.mark.parametrize("precision", [0, 1])
def test_backward_facing_step_matches_oracle(precision):
    """The backward-facing-step stand-in (Section 5.3 workloads; prescribed parabolic outflow in
    place of the do-nothing condition) on a red-refined non-convex hierarchy with greedy colouring."""
    import paper_2303_06762_gb300 as hdg
    from workloads.mesh2d import step_channel_hierarchy
    from workloads.manufactured import step_channel_velocity_2d
    from _util import topo_of
    ms = step_channel_hierarchy(4)
    ts = [topo_of(m) for m in ms]
    ps = [m.parent for m in ms]
    m, k, gamma = ms[-1], 2, 100.0
    data = dirichlet_facet_data(m.coords, m.cells, k, step_channel_velocity_2d())
    zero = np.zeros((m.n_cells, (k + 2) * (k + 3) // 2, 2))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    F = hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=0.0, gamma=gamma, precision=precision,
                                         dirichlet=torch.tensor(data, device=DEV)),
                         torch.tensor(zero, device=DEV))
    oh = HDG(ts[-1], k, nu=1.0, beta=0.0, gamma=gamma, dirichlet=data)
    Fo = oh.load(zero)
    assert rel(F.cpu().numpy(), Fo) < 1e-12
    ud, pd = oh.solve_direct(Fo)
    o = parity_opts(hdg, gamma)
    o.floor_rel = 1e-13          # |F| carries the AL coupling of the in- and outflow fluxes
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    eu, ep = relnorm(u.cpu().numpy(), ud), relnorm(p.cpu().numpy(), pd)
    print(f"step, precision {precision}: its {info['krylov_its']} vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-8 and ep < 1e-8 and info["div_l2"] < 1e-8
    if precision == 0:
        M = build_hpmg(ts, ps, k, 1.0, 0.0, gamma, hdg_k=oh)
        ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, Fo, M, bflux=oh.boundary_flux())
        u, p, info = hdg.hdg_solve(ctx, F)
        assert info["krylov_its"] == ro.krylov_its
        assert relnorm(u.cpu().numpy(), ro.u) < 1e-10
