"""GPU parity: every step of the hot path through the C ABI against the CPU oracle.

Sizes span several levels, ragged boundary patches and both structured and
jittered / orientation-shuffled meshes.  FP64 steps must agree with the oracle
to round-off (1e-12 relative for one-shot operators, 1e-10 for iterated ones);
full solves must take the same number of iterations; the mixed-precision
solve must reach the exact discrete solution to the solver tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d, unit_square_hierarchy
from oracle.hdg import HDG
from oracle.mg import (BlockGS, vertex_patches, averaging_prolongation, interior_fine_dofs,
                       harmonic_prolongation, build_hpmg, Level, MGh)
from oracle.krylov import uzawa
from _util import hierarchy, forcing, topo_of, rel, relnorm, parity_opts

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _hdg():
    import paper_2303_06762_gb300 as hdg
    return hdg


def setup_case(N0, nl, k, gamma=100.0, beta=1.0, nu=1.0, precision=0, fused=0, **meshkw):
    hdg = _hdg()
    ms, ts, ps = hierarchy(N0, nl, **meshkw)
    fv = forcing(ms[-1], k, curl_bubble_2d(), nu, beta)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=nu, beta=beta, gamma=gamma, precision=precision,
                     fused_coarse_cells=fused)
    F = hdg.hdg_condense(ctx, prm, torch.tensor(fv, device=DEV))
    return ms, ts, ps, fv, ctx, F


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


MESHES = [dict(), dict(shuffle_seed=7), dict(jitter=0.25, seed=3, shuffle_seed=5)]


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mesh", range(len(MESHES)))
def test_element_matrices_and_load(k, mesh):
    hdg = _hdg()
    nu, beta, gamma = 1.3, 0.7, 50.0
    ms, ts, ps, fv, ctx, F = setup_case(2, 2, k, gamma=gamma, beta=beta, nu=nu, **MESHES[mesh])
    oh = HDG(ts[-1], k, nu=nu, beta=beta, gamma=gamma)
    A = host(hdg.hdg_get_element_matrices(ctx, -1))
    Ao = np.stack([oh.element_matrix(c) for c in range(ts[-1].n_cells)])
    assert rel(A, Ao) < 1e-12
    assert rel(host(F), oh.load(fv)) < 1e-12
    for l in range(len(ts)):
        A0 = host(hdg.hdg_get_element_matrices(ctx, l))
        o0 = HDG(ts[l], 0, nu=nu, beta=beta, gamma=gamma)
        assert rel(A0, np.stack([o0.element_matrix(c) for c in range(ts[l].n_cells)])) < 1e-12


@pytest.mark.parametrize("k", [0, 2, 3])
def test_apply(k):
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, k, shuffle_seed=3)
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    x = np.random.default_rng(1).standard_normal(oh.n_dof)
    y = host(hdg.hdg_apply(ctx, dev(x)))
    assert rel(y, oh.matrix() @ x) < 1e-13
    for l in range(3):
        o0 = HDG(ts[l], 0, gamma=100.0, beta=1.0)
        x0 = np.random.default_rng(l).standard_normal(o0.n_dof)
        assert rel(host(hdg.hdg_level_apply(ctx, l, dev(x0))), o0.matrix() @ x0) < 1e-13


@pytest.mark.parametrize("level", [-1, 1, 2])
@pytest.mark.parametrize("reverse", [False, True])
def test_block_gs_sweep(level, reverse):
    hdg = _hdg()
    k = 2
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, k, jitter=0.2, seed=1)
    t = ts[-1] if level < 0 else ts[level]
    oh = HDG(t, k if level < 0 else 0, gamma=100.0, beta=1.0)
    gs = BlockGS(oh.matrix(), vertex_patches(t, oh.dpf))
    rng = np.random.default_rng(2)
    g, u0 = rng.standard_normal((2, oh.n_dof))
    uo = (gs.backward if reverse else gs.forward)(g, u0.copy())
    ud = dev(u0)
    hdg.hdg_smooth(ctx, level, dev(g), ud, 1, reverse)
    assert rel(host(ud), uo) < 1e-11


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("mesh", [0, 2])
def test_block_gs_sweep_mixed_order_k(k, mesh):
    """The FP32 order-k sweep (bulk-copy staged where the patch sizes allow) against the
    oracle's sequential block GS."""
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, k, precision=hdg.HDG_MIXED_FP32, **MESHES[mesh])
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    gs = BlockGS(oh.matrix(), vertex_patches(oh.topo, oh.dpf))
    rng = np.random.default_rng(12)
    for reverse in (False, True):
        g, u0 = rng.standard_normal((2, oh.n_dof))
        uo = (gs.backward if reverse else gs.forward)(g, u0.copy())
        ud = dev(u0)
        hdg.hdg_smooth(ctx, -1, dev(g), ud, 1, reverse)
        assert rel(host(ud), uo) < 2e-5


def test_transfers_and_coarse_solve():
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, 1, jitter=0.3, seed=2, shuffle_seed=1)
    for l in (1, 2):
        Af = HDG(ts[l], 0, gamma=100.0, beta=1.0).matrix()
        P = harmonic_prolongation(Af, averaging_prolongation(ts[l - 1], ts[l], ps[l]),
                                  interior_fine_dofs(ts[l], ps[l]))
        rng = np.random.default_rng(l)
        uc = rng.standard_normal(P.shape[1])
        uf0 = rng.standard_normal(P.shape[0])
        ufd = dev(uf0)
        hdg.hdg_prolong_add(ctx, l, dev(uc), ufd)
        assert rel(host(ufd) - uf0, P @ uc) < 1e-12
        rf = rng.standard_normal(P.shape[0])
        assert rel(host(hdg.hdg_restrict(ctx, l, dev(rf))), P.T @ rf) < 1e-12
    A0 = HDG(ts[0], 0, gamma=100.0, beta=1.0).matrix().toarray()
    g = np.random.default_rng(9).standard_normal(A0.shape[0])
    assert rel(host(hdg.hdg_coarse_solve(ctx, dev(g))), np.linalg.solve(A0, g)) < 1e-11


def _oracle_mg(ts, ps, k, gamma, beta=1.0, q=1):
    return build_hpmg(ts, ps, k, 1.0, beta, gamma, q=q)


@pytest.mark.parametrize("q", [1, 2])
@pytest.mark.parametrize("fused", [0, 2048])
def test_mg_h_and_mg_hp(q, fused):
    hdg = _hdg()
    k = 2
    ms, ts, ps, fv, ctx, F = setup_case(2, 4, k, shuffle_seed=11)
    hdg.hdg_condense(ctx, hdg.Params(k=k, beta=1.0, gamma=100.0, cycle=q, fused_coarse_cells=fused))
    M = _oracle_mg(ts, ps, k, 100.0, q=q)
    rng = np.random.default_rng(4)
    g0 = rng.standard_normal(2 * ts[-1].n_interior)
    assert rel(host(hdg.hdg_mg_h(ctx, dev(g0))), M.mgh(g0, 1, q)) < 1e-10
    r = rng.standard_normal(M.A.shape[0])
    assert rel(host(hdg.hdg_precond_apply(ctx, dev(r))), M(r)) < 1e-10


def test_mg_hp_k0_is_mg_h():
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, 0)
    r = np.random.default_rng(5).standard_normal(2 * ts[-1].n_interior)
    a = host(hdg.hdg_precond_apply(ctx, dev(r)))
    b = host(hdg.hdg_mg_h(ctx, dev(r)))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("k,gamma,mesh", [(1, 1e2, 0), (2, 1e2, 1), (3, 1e4, 2), (0, 1e2, 0)])
def test_solve_matches_oracle(k, gamma, mesh):
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 3, k, gamma=gamma, **MESHES[mesh])
    oh = HDG(ts[-1], k, gamma=gamma, beta=1.0)
    M = build_hpmg(ts, ps, k, 1.0, 1.0, gamma, hdg_k=oh)
    Fo = oh.load(fv)
    ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, Fo, M)
    u, p, info = hdg.hdg_solve(ctx, F)
    # the same iteration as the oracle's (default stopping rule): same counts, same iterates
    assert info["krylov_its"] == ro.krylov_its
    eu, ep = relnorm(host(u), ro.u), relnorm(host(p), ro.p)
    print(f"k={k} gamma={gamma:g}: vs oracle iteration |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-10
    # at gamma = 1e4 the last inner solves stop on the residual floor, where the pressure
    # update eps^-1 div u magnifies rounding-order differences of u (Remark 3.1)
    assert ep < (1e-10 if gamma <= 1e2 else 5e-9)
    # against the exact discrete solution (sparse direct solve of the condensed saddle point)
    # with the parity stopping rule
    ud, pd = oh.solve_direct(Fo)
    u, p, info = hdg.hdg_solve(ctx, F, opts=parity_opts(hdg, gamma))
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"k={k} gamma={gamma:g}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-10
    assert ep < (1e-10 if gamma <= 1e2 else 5e-9)


@pytest.mark.parametrize("k", [1, 3])
def test_mixed_precision_solve(k):
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(2, 4, k, gamma=100.0, precision=hdg.HDG_MIXED_FP32)
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    ud, pd = oh.solve_direct(oh.load(fv))
    u, p, info = hdg.hdg_solve(ctx, F)
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"mixed k={k}: vs direct |du| {eu:.2e} |dp| {ep:.2e} (default stopping rule)")
    assert eu < 1e-8 and ep < 1e-8
    assert info["krylov_its_total"] > 0
    # the FP64 outer iteration reaches the FP64 target with the parity stopping rule
    u, p, info = hdg.hdg_solve(ctx, F, opts=parity_opts(hdg, 100.0))
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"mixed k={k}: vs direct |du| {eu:.2e} |dp| {ep:.2e} (parity stopping rule)")
    assert eu < 1e-10 and ep < 1e-9


def test_single_level_and_coarsest_one_square():
    hdg = _hdg()
    ms, ts, ps, fv, ctx, F = setup_case(4, 1, 2)       # one level: MG_h is the coarse solve
    oh = HDG(ts[0], 2, gamma=100.0, beta=1.0)
    u, p, info = hdg.hdg_solve(ctx, F)
    ud, pd = oh.solve_direct(oh.load(fv))
    assert relnorm(host(u), ud) < 1e-8 and relnorm(host(p), pd) < 1e-8
    ms, ts, ps, fv, ctx, F = setup_case(1, 4, 1)       # coarsest mesh: 2 cells, 1 interior facet
    oh = HDG(ts[-1], 1, gamma=100.0, beta=1.0)
    M = build_hpmg(ts, ps, 1, 1.0, 1.0, 100.0, hdg_k=oh)
    r = np.random.default_rng(0).standard_normal(oh.n_dof)
    assert rel(host(hdg.hdg_precond_apply(ctx, dev(r))), M(r)) < 1e-10


def test_error_paths():
    hdg = _hdg()
    ms, ts, ps = hierarchy(2, 2)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    x = torch.zeros(10, dtype=torch.float64, device=DEV)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_apply(ctx, x)
    assert e.value.status == 9          # operator used before hdg_condense
    for bad in (dict(k=5), dict(nu=0.0), dict(gamma=-1.0), dict(cycle=3), dict(m_p=0)):
        with pytest.raises(hdg.HdgError) as e:
            hdg.hdg_condense(ctx, hdg.Params(**{**dict(k=1), **bad}))
        assert e.value.status == 1
    bad_parent = [m for m in ms]
    bad_parent[1].parent = np.zeros_like(bad_parent[1].parent)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_setup_mesh_hierarchy(bad_parent)
    assert e.value.status == 1


def test_full_size_sampled_parity():
    """512x512 triangulation, k = 3 (the benchmark configuration): sampled cells'
    condensed matrices and loads against the oracle computed cell by cell, and
    sampled rows of the operator apply."""
    hdg = _hdg()
    from oracle.spaces import Element
    from oracle.hdg import condense_cell
    from workloads import forcing_at_lattice
    k, nu, beta, gamma = 3, 1.0, 1.0, 100.0
    ms = unit_square_hierarchy(8, 7)            # 8 .. 512
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(nu, beta))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=k, nu=nu, beta=beta, gamma=gamma), dev(fv))
    A = hdg.hdg_get_element_matrices(ctx, -1)
    rng = np.random.default_rng(123)
    cells = rng.choice(fine.n_cells, 48, replace=False)
    for c in cells:
        gv = fine.cells[c]
        X = fine.coords[gv]
        cc = condense_cell(Element(X - X[0], gv, k), nu, beta)
        d = cc.d
        Ao = cc.A + (gamma * nu / cc.area) * np.outer(d, d)
        assert rel(host(A[c]), Ao) < 1e-11
    s = ctx.sizes()
    x = rng.standard_normal(s.n_dof)
    y = host(hdg.hdg_apply(ctx, dev(x)))
    # rows of sampled interior facets from the two adjacent cells' oracle matrices
    from oracle.topology import build_topology
    topo = build_topology(fine.coords, fine.cells, fine.vertex_colour)
    dpf = 2 * (k + 1)
    for i in rng.choice(topo.n_interior, 24, replace=False):
        F = topo.interior_facets[i]
        acc = np.zeros(dpf)
        for c in topo.facet_cells[F]:
            gv = fine.cells[c]
            X = fine.coords[gv]
            cc = condense_cell(Element(X - X[0], gv, k), nu, beta)
            Ao = cc.A + (gamma * nu / cc.area) * np.outer(cc.d, cc.d)
            xl = np.zeros(3 * dpf)
            for f in range(3):
                j = topo.interior_index[topo.cell_facets[c, f]]
                if j >= 0:
                    xl[f * dpf:(f + 1) * dpf] = x[j * dpf:(j + 1) * dpf]
            lf = list(topo.cell_facets[c]).index(F)
            acc += Ao[lf * dpf:(lf + 1) * dpf] @ xl
        assert rel(y[i * dpf:(i + 1) * dpf], acc) < 1e-11


_BIG_ORACLE = {}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("fused", [512, 2048])
def test_mg_h_fused_and_multiblock_levels(precision, fused):
    """Hierarchy 4x4..128x128 with the fused kernel on levels up to 16x16 (one block, level
    vectors in shared memory) or 32x32 (a cluster) and the multi-block kernels above:
    MG_h and MG_hp against the oracle."""
    hdg = _hdg()
    k = 1
    ms, ts, ps, fv, ctx, F = setup_case(4, 6, k, precision=precision, fused=fused)
    if "M" not in _BIG_ORACLE:
        _BIG_ORACLE["M"] = _oracle_mg(ts, ps, k, 100.0)
    M = _BIG_ORACLE["M"]
    rng = np.random.default_rng(8)
    g0 = rng.standard_normal(2 * ts[-1].n_interior)
    tol = 1e-10 if precision == 0 else 1e-4
    assert rel(host(hdg.hdg_mg_h(ctx, dev(g0))), M.mgh(g0, 1, 1)) < tol
    r = rng.standard_normal(M.A.shape[0])
    assert rel(host(hdg.hdg_precond_apply(ctx, dev(r))), M(r)) < tol
