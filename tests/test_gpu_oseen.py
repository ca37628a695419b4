"""GPU parity of the Oseen path (Section 4): upwind convection in the condensed
operator, the hp-multigrid built on it, the Uzawa/FGMRES solve and the adjoint
with the transposed convection, all through the C ABI against the CPU oracle.

The convecting field is the curl of the continuous degree-(k+1) interpolant of
psi = c sin²(pi x) sin²(pi y) (max|b| = 1), sampled at each cell's lattice.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d, forcing_at_lattice
from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
from oracle.hdg import HDG
from oracle.mg import (BlockGS, vertex_patches, averaging_prolongation, interior_fine_dofs,
                       harmonic_prolongation, build_hpmg, lowest_order_convection)
from oracle.krylov import uzawa
from oracle.adjoint import objective_and_gradient
from _util import hierarchy, rel, relnorm, parity_opts

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PSI, B = convecting_stream_2d(1.0)
SOL = curl_bubble_2d()


def _hdg():
    import paper_2303_06762_gb300 as hdg
    return hdg


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def oseen_case(N0, nl, k, Re=100.0, gamma=100.0, beta=0.0, precision=0, fused=0, nu_elem=None, **meshkw):
    hdg = _hdg()
    ms, ts, ps = hierarchy(N0, nl, **meshkw)
    nu = 1.0 / Re
    conv = curl_lattice_2d(ms[-1].coords, ms[-1].cells, k + 1, PSI)
    fv = forcing_at_lattice(ms[-1].coords, ms[-1].cells, k, SOL.forcing(nu, beta, conv=B))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=nu, beta=beta, gamma=gamma, precision=precision, fused_coarse_cells=fused,
                     conv=dev(conv), nu_elem=None if nu_elem is None else dev(nu_elem))
    F = hdg.hdg_condense(ctx, prm, dev(fv))
    return ms, ts, ps, conv, fv, ctx, F, nu


MESHES = [dict(), dict(shuffle_seed=7), dict(jitter=0.25, seed=3, shuffle_seed=5)]


@pytest.mark.parametrize("k", [1, 3])
def test_transposed_apply(k):
    """hdg_apply_transpose against the transposed oracle matrices, on the order-k level and
    the lowest-order levels of the Oseen operator."""
    hdg = _hdg()
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 3, k, Re=50.0, **MESHES[2])
    oh = HDG(ts[-1], k, nu=nu, gamma=100.0, conv=conv)
    x = np.random.default_rng(k).standard_normal(oh.n_dof)
    A = oh.matrix()
    y = host(hdg.hdg_apply_transpose(ctx, dev(x)))
    assert rel(y, A.T @ x) < 1e-13
    assert rel(y, A @ x) > 1e-6            # the Oseen operator is not symmetric
    cl = lowest_order_convection(ts, ps, conv)
    for l in range(len(ts)):
        o0 = HDG(ts[l], 0, nu=nu, gamma=100.0, conv=cl[l])
        x0 = np.random.default_rng(l).standard_normal(o0.n_dof)
        assert rel(host(hdg.hdg_apply_transpose(ctx, dev(x0), level=l)), o0.matrix().T @ x0) < 1e-13


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mesh", [0, 2])
def test_oseen_element_matrices_and_load(k, mesh):
    hdg = _hdg()
    gamma, beta = 50.0, 0.5
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 2, k, Re=10.0, gamma=gamma, beta=beta, **MESHES[mesh])
    oh = HDG(ts[-1], k, nu=nu, beta=beta, gamma=gamma, conv=conv)
    A = host(hdg.hdg_get_element_matrices(ctx, -1))
    Ao = np.stack([oh.element_matrix(c) for c in range(ts[-1].n_cells)])
    assert np.abs(Ao - np.transpose(Ao, (0, 2, 1))).max() > 1e-3 * np.abs(Ao).max()
    assert rel(A, Ao) < 1e-12
    assert rel(host(F), oh.load(fv)) < 1e-12
    cl = lowest_order_convection(ts, ps, conv)
    for l in range(len(ts)):
        A0 = host(hdg.hdg_get_element_matrices(ctx, l))
        o0 = HDG(ts[l], 0, nu=nu, beta=beta, gamma=gamma, conv=cl[l])
        assert rel(A0, np.stack([o0.element_matrix(c) for c in range(ts[l].n_cells)])) < 1e-12


@pytest.mark.parametrize("k", [1, 3])
def test_oseen_apply_smoother_transfers(k):
    hdg = _hdg()
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 3, k, shuffle_seed=3)
    cl = lowest_order_convection(ts, ps, conv)
    oh = HDG(ts[-1], k, nu=nu, gamma=100.0, conv=conv)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(oh.n_dof)
    assert rel(host(hdg.hdg_apply(ctx, dev(x))), oh.matrix() @ x) < 1e-13
    levels = [HDG(ts[l], 0, nu=nu, gamma=100.0, conv=cl[l]) for l in range(3)]
    for l, o0 in enumerate(levels):
        x0 = rng.standard_normal(o0.n_dof)
        assert rel(host(hdg.hdg_level_apply(ctx, l, dev(x0))), o0.matrix() @ x0) < 1e-13
    for level, o in ((-1, oh), (2, levels[2]), (1, levels[1])):
        gs = BlockGS(o.matrix(), vertex_patches(o.topo, o.dpf))
        for reverse in (False, True):
            g, u0 = rng.standard_normal((2, o.n_dof))
            uo = (gs.backward if reverse else gs.forward)(g, u0.copy())
            ud = dev(u0)
            hdg.hdg_smooth(ctx, level, dev(g), ud, 1, reverse)
            assert rel(host(ud), uo) < 1e-11
    for l in (1, 2):
        P = harmonic_prolongation(levels[l].matrix(), averaging_prolongation(ts[l - 1], ts[l], ps[l]),
                                  interior_fine_dofs(ts[l], ps[l]))
        uc = rng.standard_normal(P.shape[1])
        uf0 = rng.standard_normal(P.shape[0])
        ufd = dev(uf0)
        hdg.hdg_prolong_add(ctx, l, dev(uc), ufd)
        assert rel(host(ufd) - uf0, P @ uc) < 1e-12
        rf = rng.standard_normal(P.shape[0])
        assert rel(host(hdg.hdg_restrict(ctx, l, dev(rf))), P.T @ rf) < 1e-12
    A0 = levels[0].matrix().toarray()
    g = rng.standard_normal(A0.shape[0])
    assert rel(host(hdg.hdg_coarse_solve(ctx, dev(g))), np.linalg.solve(A0, g)) < 1e-11


@pytest.mark.parametrize("fused", [0, 2048])
def test_oseen_mg_h_and_mg_hp(fused):
    hdg = _hdg()
    k = 2
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 4, k, Re=100.0, fused=fused, shuffle_seed=11)
    M = build_hpmg(ts, ps, k, nu, 0.0, 100.0, conv=conv)
    rng = np.random.default_rng(4)
    g0 = rng.standard_normal(2 * ts[-1].n_interior)
    assert rel(host(hdg.hdg_mg_h(ctx, dev(g0))), M.mgh(g0, 1, 1)) < 1e-10
    r = rng.standard_normal(M.A.shape[0])
    assert rel(host(hdg.hdg_precond_apply(ctx, dev(r))), M(r)) < 1e-10


@pytest.mark.parametrize("k,Re,mesh", [(1, 1.0, 0), (2, 100.0, 1), (2, 100.0, 2)])
def test_oseen_solve_matches_oracle(k, Re, mesh):
    hdg = _hdg()
    gamma = 100.0
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 3, k, Re=Re, gamma=gamma, **MESHES[mesh])
    M = build_hpmg(ts, ps, k, nu, 0.0, gamma, conv=conv)
    oh = M.hdg
    Fo = oh.load(fv)
    ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, Fo, M)
    u, p, info = hdg.hdg_solve(ctx, F)
    assert info["krylov_its"] == ro.krylov_its
    eu, ep = relnorm(host(u), ro.u), relnorm(host(p), ro.p)
    print(f"Oseen k={k} Re={Re:g}: vs oracle iteration |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-10 and ep < 1e-10
    ud, pd = oh.solve_direct(Fo)
    u, p, info = hdg.hdg_solve(ctx, F, opts=parity_opts(hdg, gamma))
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"Oseen k={k} Re={Re:g}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    # nu = 1/Re scales the load and the pressure differently from the Stokes cases; the
    # parity rule's floor leaves the pressure a few 1e-10 from the direct solve at Re = 100
    assert eu < 1e-9 and ep < 1e-9


def test_oseen_restart_50_matches_oracle():
    """The Oseen configuration's FGMRES(50) (restart lengths up to 64 in single-load solves)."""
    hdg = _hdg()
    k, gamma = 2, 100.0
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 3, k, Re=100.0, gamma=gamma)
    M = build_hpmg(ts, ps, k, nu, 0.0, gamma, conv=conv)
    oh = M.hdg
    ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, oh.load(fv), M, restart=50)
    o = hdg.default_solve_opts()
    o.restart = 50
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    assert info["krylov_its"] == ro.krylov_its
    assert relnorm(host(u), ro.u) < 1e-10 and relnorm(host(p), ro.p) < 1e-10
    o.restart = 65
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_solve(ctx, F, opts=o)
    assert e.value.status == 1


def test_oseen_mixed_precision_solve():
    hdg = _hdg()
    k = 2
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 4, k, Re=100.0, precision=1)
    oh = HDG(ts[-1], k, nu=nu, gamma=100.0, conv=conv)
    ud, pd = oh.solve_direct(oh.load(fv))
    u, p, info = hdg.hdg_solve(ctx, F)
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"Oseen mixed: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-8 and ep < 1e-8


@pytest.mark.parametrize("k,Re", [(1, 1.0), (2, 100.0)])
def test_oseen_adjoint_gradients(k, Re):
    hdg = _hdg()
    rng = np.random.default_rng(7)
    ms, ts, ps = hierarchy(2, 3, shuffle_seed=4)
    nu_e = (1.0 / Re) * (1 + 0.1 * rng.uniform(-1, 1, ms[-1].n_cells))
    ms, ts, ps, conv, fv, ctx, F, nu = oseen_case(2, 3, k, Re=Re, nu_elem=nu_e, shuffle_seed=4)
    fine = ms[-1]
    ut = forcing_at_lattice(fine.coords, fine.cells, k, SOL.u) + 0.1 * rng.standard_normal(fv.shape)
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    A_before = host(hdg.hdg_get_element_matrices(ctx, -1))
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    J, gf, gn, info_a = hdg.hdg_adjoint(ctx, dev(fv), u, dev(ut), opts=o)
    Jo, gfo, gno, *_ = objective_and_gradient(ts[-1], k, fv, ut, nu_e, conv=conv)
    assert abs(J - Jo) < 1e-9 * Jo
    assert rel(host(gf), gfo) < 1e-7
    assert rel(host(gn), gno) < 1e-7
    # the primal operators are back after the transposed adjoint solve
    assert np.array_equal(host(hdg.hdg_get_element_matrices(ctx, -1)), A_before)


def test_full_size_oseen_sampled_parity():
    """The Oseen benchmark configuration (128x128, k = 2, Re = 100): sampled cells' condensed matrices
    against the oracle computed cell by cell."""
    from oracle.spaces import Element
    from oracle.hdg import condense_cell
    from workloads import unit_square_hierarchy
    hdg = _hdg()
    k, Re, gamma = 2, 100.0, 100.0
    nu = 1.0 / Re
    ms = unit_square_hierarchy(8, 5)            # 8 .. 128
    fine = ms[-1]
    conv = curl_lattice_2d(fine.coords, fine.cells, k + 1, PSI)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=k, nu=nu, beta=0.0, gamma=gamma, conv=dev(conv)))
    A = hdg.hdg_get_element_matrices(ctx, -1)
    rng = np.random.default_rng(17)
    for c in rng.choice(fine.n_cells, 40, replace=False):
        gv = fine.cells[c]
        X = fine.coords[gv]
        cc = condense_cell(Element(X - X[0], gv, k), nu, 0.0, conv[c])
        Ao = cc.A + (gamma * nu / cc.area) * np.outer(cc.d, cc.d)
        assert rel(host(A[c]), Ao) < 1e-11
