"""GPU parity of the multi-right-hand-side (batched) forms: hdg_apply_multi,
hdg_precond_apply_multi and hdg_solve_multi against the single-load forms
column by column and against the oracle's exact solution.

Loads follow the many-right-hand-side workload: seeded sums of Fourier modes
plus gradient fields (workloads.manufactured.fourier_forcing_2d).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import forcing_at_lattice
from workloads.manufactured import fourier_forcing_2d, convecting_stream_2d, curl_lattice_2d
from oracle.hdg import HDG
from _util import hierarchy, rel, relnorm

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _hdg():
    import paper_2303_06762_gb300 as hdg
    return hdg


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _opts(hdg):
    # one decade below the default stopping rule, so that the solution (not only the
    # residual) is within 1e-8 of the exact discrete solution for these rough loads
    o = hdg.default_solve_opts()
    o.rtol, o.floor_rel, o.uzawa_tol = 1e-10, 1e-11, 1e-10
    return o


def _setup(N0, nl, k, nrhs, precision=0, gamma=100.0, beta=1.0, nu=1.0, conv=False, **meshkw):
    hdg = _hdg()
    ms, ts, ps = hierarchy(N0, nl, **meshkw)
    fine = ms[-1]
    fvs = [forcing_at_lattice(fine.coords, fine.cells, k, fourier_forcing_2d(j)) for j in range(nrhs)]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    cv = None
    if conv:
        psi, _ = convecting_stream_2d(1.0)
        cv = curl_lattice_2d(fine.coords, fine.cells, k + 1, psi)
    prm = hdg.Params(k=k, nu=nu, beta=beta, gamma=gamma, precision=precision,
                     conv=None if cv is None else dev(cv))
    hdg.hdg_condense(ctx, prm)
    F = torch.stack([hdg.hdg_load(ctx, dev(fv)) for fv in fvs])
    return ms, ts, ps, fvs, ctx, F, cv


@pytest.mark.parametrize("nrhs", [1, 3, 8])
@pytest.mark.parametrize("precision", [0, 1])
def test_apply_and_precond_multi_match_single(nrhs, precision):
    hdg = _hdg()
    ms, ts, ps, fvs, ctx, F, _ = _setup(2, 3, 2, nrhs, precision=precision, shuffle_seed=3)
    gen = torch.Generator(device=DEV).manual_seed(17 + nrhs)
    X = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    Y = hdg.hdg_apply_multi(ctx, X)
    Z = hdg.hdg_precond_apply_multi(ctx, X)
    for r in range(nrhs):
        assert rel(host(Y[r]), host(hdg.hdg_apply(ctx, X[r].contiguous()))) < 1e-14
        zs = host(hdg.hdg_precond_apply(ctx, X[r].contiguous()))
        # FP32: the batched and the single-load sweeps sum in different orders (2e-5, the
        # FP32 sweep's own parity bound)
        assert rel(host(Z[r]), zs) < (1e-12 if precision == 0 else 2e-5)


@pytest.mark.parametrize("k,nrhs,precision,mesh", [(1, 4, 0, {}), (2, 5, 1, dict(shuffle_seed=2)),
                                                   (3, 8, 1, dict(jitter=0.2, seed=1))])
def test_solve_multi_matches_single_and_direct(k, nrhs, precision, mesh):
    hdg = _hdg()
    ms, ts, ps, fvs, ctx, F, _ = _setup(2, 3, k, nrhs, precision=precision, **mesh)
    U, P, infos = hdg.hdg_solve_multi(ctx, F, opts=_opts(hdg))
    oh = HDG(ts[-1], k, nu=1.0, beta=1.0, gamma=100.0)
    for r in range(nrhs):
        u1, p1, info1 = hdg.hdg_solve(ctx, F[r].contiguous(), opts=_opts(hdg))
        if precision == 0:
            assert infos[r]["krylov_its"] == info1["krylov_its"]
            assert rel(host(U[r]), host(u1)) < 1e-9
        else:
            assert abs(infos[r]["krylov_its_total"] - info1["krylov_its_total"]) <= infos[r]["uzawa_its"]
        ud, pd = oh.solve_direct(oh.load(fvs[r]))
        eu, ep = relnorm(host(U[r]), ud), relnorm(host(P[r]), pd)
        print(f"batched k={k} column {r}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
        assert eu < 1e-8 and ep < 1e-8


def test_solve_multi_oseen_and_wide_batch():
    hdg = _hdg()
    nrhs = 64
    ms, ts, ps, fvs, ctx, F, cv = _setup(4, 2, 3, nrhs, precision=1, nu=0.01, beta=0.0, conv=True)
    U, P, infos = hdg.hdg_solve_multi(ctx, F, opts=_opts(hdg))
    oh = HDG(ts[-1], 3, nu=0.01, beta=0.0, gamma=100.0, conv=cv)
    for r in (0, 17, 63):
        ud, pd = oh.solve_direct(oh.load(fvs[r]))
        eu, ep = relnorm(host(U[r]), ud), relnorm(host(P[r]), pd)
        print(f"batched Oseen column {r}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
        assert eu < 1e-8 and ep < 1e-8
    assert all(i["uzawa_its"] >= 1 for i in infos)


def test_multi_error_paths():
    hdg = _hdg()
    ms, ts, ps, fvs, ctx, F, _ = _setup(2, 2, 1, 2)
    lib = hdg.load_library()
    assert lib.hdg_apply_multi(ctx.handle, 0, None, None, None) == 1
    assert lib.hdg_apply_multi(ctx.handle, 65, None, None, None) == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_batched_uneven_meshes(precision):
    """Several meshes of different sizes solved concurrently equal their separate solves."""
    from workloads import curl_bubble_2d
    hdg = _hdg()
    k = 2
    ctxs, Fs, ohs, fvs = [], [], [], []
    for N0, nl in ((2, 2), (3, 2), (2, 3)):
        ms, ts, ps = hierarchy(N0, nl)
        fine = ms[-1]
        fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(1.0, 1.0))
        ctx = hdg.hdg_setup_mesh_hierarchy(ms)
        Fs.append(hdg.hdg_condense(ctx, hdg.Params(k=k, beta=1.0, gamma=100.0, precision=precision), dev(fv)))
        ctxs.append(ctx)
        ohs.append(HDG(ts[-1], k, nu=1.0, beta=1.0, gamma=100.0))
        fvs.append(fv)
    us, ps_, infos, stat = hdg.hdg_solve_batched(ctxs, Fs)
    assert stat == [0, 0, 0]
    for ctx, F, u, p, info, oh, fv in zip(ctxs, Fs, us, ps_, infos, ohs, fvs):
        u1, p1, info1 = hdg.hdg_solve(ctx, F)
        assert info["krylov_its"] == info1["krylov_its"]
        assert rel(host(u), host(u1)) < 1e-13
        ud, pd = oh.solve_direct(oh.load(fv))
        eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
        print(f"uneven meshes: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
        assert eu < 1e-8 and ep < 1e-8
    lib = hdg.load_library()
    import ctypes
    same = (ctypes.c_void_p * 2)(ctxs[0].handle, ctxs[0].handle)
    assert lib.hdg_solve_batched(ctypes.cast(same, ctypes.c_void_p), 2, None, None, None, None, None, None) == 1


def test_full_size_batched_sampled_parity():
    """The batched benchmark configuration (256x256, k = 3, 64 loads): sampled rows of the batched
    operator apply against the oracle's condensed cell matrices computed one by one, and two columns of
    the batched preconditioner against single-column applications."""
    from oracle.spaces import Element
    from oracle.hdg import condense_cell
    from oracle.topology import build_topology
    from workloads import unit_square_hierarchy
    hdg = _hdg()
    k, nu, beta, gamma, R = 3, 1.0, 1.0, 100.0, 64
    ms = unit_square_hierarchy(8, 6)            # 8 .. 256
    fine = ms[-1]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=k, nu=nu, beta=beta, gamma=gamma, precision=1))
    s = ctx.sizes()
    rng = np.random.default_rng(5)
    X = torch.tensor(rng.standard_normal((R, s.n_dof)), device=DEV)
    Y = host(hdg.hdg_apply_multi(ctx, X))
    Xh = host(X)
    topo = build_topology(fine.coords, fine.cells, fine.vertex_colour)
    dpf = 2 * (k + 1)
    for i in rng.choice(topo.n_interior, 12, replace=False):
        F = topo.interior_facets[i]
        acc = np.zeros((dpf, R))
        for c in topo.facet_cells[F]:
            gv = fine.cells[c]
            X0 = fine.coords[gv]
            cc = condense_cell(Element(X0 - X0[0], gv, k), nu, beta)
            Ao = cc.A + (gamma * nu / cc.area) * np.outer(cc.d, cc.d)
            xl = np.zeros((3 * dpf, R))
            for f in range(3):
                j = topo.interior_index[topo.cell_facets[c, f]]
                if j >= 0:
                    xl[f * dpf:(f + 1) * dpf] = Xh[:, j * dpf:(j + 1) * dpf].T
            lf = list(topo.cell_facets[c]).index(F)
            acc += Ao[lf * dpf:(lf + 1) * dpf] @ xl
        assert rel(Y[:, i * dpf:(i + 1) * dpf].T, acc) < 1e-11
    # FP32 preconditioner: the batched and single kernels sum in different orders, and
    # six levels of V-cycle amplify the FP32 rounding differences to about 1e-5
    Z = hdg.hdg_precond_apply_multi(ctx, X)
    for r in (0, 63):
        assert rel(host(Z[r]), host(hdg.hdg_precond_apply(ctx, X[r].contiguous()))) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_tile_autotuner(precision):
    """The autotuner returns one of the candidate tiles, and every tile of the batched
    order-k sweep gives bitwise the same preconditioner."""
    hdg = _hdg()
    ms, ts, ps, fvs, ctx, F, _ = _setup(2, 3, 3, 8, precision=precision, shuffle_seed=5)
    gen = torch.Generator(device=DEV).manual_seed(2)
    X = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    rb, nt, t = hdg.hdg_tune_batched(ctx, 8)
    assert rb in (1, 2, 4) and nt in (128, 256) and t > 0
    Z = host(hdg.hdg_precond_apply_multi(ctx, X))
    for rb2 in (1, 2, 4):
        for nt2 in (128, 256):
            hdg.hdg_set_batched_tile(ctx, rb2, nt2)
            assert np.array_equal(host(hdg.hdg_precond_apply_multi(ctx, X)), Z)
    hdg.hdg_set_batched_tile(ctx, 0, 0)
    assert np.array_equal(host(hdg.hdg_precond_apply_multi(ctx, X)), Z)
    with pytest.raises(hdg.HdgError):
        hdg.hdg_set_batched_tile(ctx, 3, 128)
