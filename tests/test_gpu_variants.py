"""GPU parity of the solver variants against the oracle: the damped block-Jacobi smoother
(eq. bjac), the additive form of Algorithm 2 (Remark 3.4) and the preconditioned conjugate
gradients of Section 5, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d
from oracle.hdg import HDG
from oracle.mg import BlockJacobi, vertex_patches, build_hpmg
from oracle.krylov import uzawa
from _util import hierarchy, forcing, rel, relnorm, parity_opts

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _case(k, nl=3, gamma=100.0, precision=0, **prm):
    import paper_2303_06762_gb300 as hdg
    ms, ts, ps = hierarchy(2, nl, shuffle_seed=5)
    fv = forcing(ms[-1], k, curl_bubble_2d(), 1.0, 1.0)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    F = hdg.hdg_condense(ctx, hdg.Params(k=k, beta=1.0, gamma=gamma, precision=precision, **prm),
                         torch.tensor(fv, device=DEV))
    return hdg, ms, ts, ps, fv, ctx, F


@pytest.mark.parametrize("level", [-1, 1, 2])
@pytest.mark.parametrize("damping", [0.5, 0.3])
def test_block_jacobi_step(level, damping):
    hdg, ms, ts, ps, fv, ctx, F = _case(2, smoother=1, jacobi_damping=damping)
    t = ts[-1] if level < 0 else ts[level]
    oh = HDG(t, 2 if level < 0 else 0, gamma=100.0, beta=1.0)
    J = BlockJacobi(oh.matrix(), vertex_patches(t, oh.dpf), damping=damping)
    rng = np.random.default_rng(3)
    g, u0 = rng.standard_normal((2, oh.n_dof))
    ud = dev(u0)
    hdg.hdg_smooth(ctx, level, dev(g), ud, 2, False)
    uo = J.forward(g, J.forward(g, u0.copy()))
    assert rel(host(ud), uo) < 1e-11


@pytest.mark.parametrize("smoother,additive", [(1, 0), (0, 1), (1, 1)])
def test_variant_preconditioners_match_oracle(smoother, additive):
    k = 2
    hdg, ms, ts, ps, fv, ctx, F = _case(k, nl=4, smoother=smoother, hp_additive=additive)
    M = build_hpmg(ts, ps, k, 1.0, 1.0, 100.0, smoother="jacobi" if smoother else "gs",
                   additive=bool(additive))
    r = np.random.default_rng(4).standard_normal(M.A.shape[0])
    assert rel(host(hdg.hdg_precond_apply(ctx, dev(r))), M(r)) < 1e-10


@pytest.mark.parametrize("k,smoother", [(1, 0), (2, 0), (2, 1)])
def test_pcg_solve_matches_oracle(k, smoother):
    hdg, ms, ts, ps, fv, ctx, F = _case(k, smoother=smoother)
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    M = build_hpmg(ts, ps, k, 1.0, 1.0, 100.0, hdg_k=oh, smoother="jacobi" if smoother else "gs")
    Fo = oh.load(fv)
    ro = uzawa(M.A, oh.flux_matrix(), oh.area, oh.eps_inv, Fo, M, krylov="pcg")
    o = hdg.default_solve_opts()
    o.krylov = 1
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    assert info["krylov_its"] == ro.krylov_its
    eu, ep = relnorm(host(u), ro.u), relnorm(host(p), ro.p)
    print(f"PCG k={k} smoother={smoother}: its {info['krylov_its']} vs oracle |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-10 and ep < 1e-10
    assert abs(info["div_l2"] - ro.div_l2) <= 0.05 * ro.div_l2 + 1e-13
    ud, pd = oh.solve_direct(Fo)
    o2 = parity_opts(hdg, 100.0)
    o2.krylov = 1
    u, p, info = hdg.hdg_solve(ctx, F, opts=o2)
    assert relnorm(host(u), ud) < 1e-10 and relnorm(host(p), pd) < 1e-10


def test_pcg_mixed_precision_reaches_discrete_solution():
    k = 3
    hdg, ms, ts, ps, fv, ctx, F = _case(k, nl=4, precision=1)
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    ud, pd = oh.solve_direct(oh.load(fv))
    o = hdg.default_solve_opts()
    o.krylov = 1
    u, p, info = hdg.hdg_solve(ctx, F, opts=o)
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"PCG mixed k=3: its {info['krylov_its']} vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-8 and ep < 1e-8


def test_variants_rejected_where_unsupported():
    hdg, ms, ts, ps, fv, ctx, F = _case(1, smoother=1)
    X = torch.zeros((2, F.numel()), dtype=torch.float64, device=DEV)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_precond_apply_multi(ctx, X)
    assert e.value.status == 8
    hdg.hdg_condense(ctx, hdg.Params(k=1, beta=1.0, gamma=100.0))
    o = hdg.default_solve_opts()
    o.krylov = 1
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_solve_multi(ctx, X, opts=o)
    assert e.value.status == 8
    o.krylov = 2
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_solve(ctx, F, opts=o)
    assert e.value.status == 1
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_condense(ctx, hdg.Params(k=1, smoother=2))
    assert e.value.status == 1
