"""GPU parity of the 16-bit preconditioner copies (HDG_MIXED_FP16, HDG_MIXED_BF16).

The order-k smoother and the residual before the hp restriction read element
matrices and patch inverses stored as power-of-two-scaled rows in binary16 or
bfloat16.  The CPU model in tests/_round16.py rounds the oracle's matrices the
same way; the device preconditioner must match that model to FP32 round-off
and differ from the unrounded oracle by the rounding itself.  Full solves still
reach the exact discrete solution, since the outer FGMRES runs on the FP64
operator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d
from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
from oracle.hdg import HDG
from oracle.mg import BlockGS, vertex_patches, build_hpmg
from _util import hierarchy, forcing, rel, relnorm
from _round16 import round_hpmg, round_hpmg_tc, stored_rows, rounded_matrix

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FMT = {2: "bf16", 3: "fp16"}


def _hdg():
    import paper_2303_06762_gb300 as hdg
    return hdg


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def case(k, precision, nl=4, oseen=False, **meshkw):
    hdg = _hdg()
    ms, ts, ps = hierarchy(2, nl, **meshkw)
    nu = 0.01 if oseen else 1.0
    beta = 0.0 if oseen else 1.0
    conv = curl_lattice_2d(ms[-1].coords, ms[-1].cells, k + 1, convecting_stream_2d(1.0)[0]) if oseen else None
    fv = forcing(ms[-1], k, curl_bubble_2d(), nu, beta)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=nu, beta=beta, gamma=100.0, precision=precision,
                     conv=None if conv is None else dev(conv))
    F = hdg.hdg_condense(ctx, prm, dev(fv))
    M = build_hpmg(ts, ps, k, nu, beta, 100.0, conv=conv)
    return ctx, F, M, fv, ts


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("k", [1, 3])
def test_order_k_sweep_matches_rounded_model(precision, k):
    hdg = _hdg()
    ctx, F, M, fv, ts = case(k, precision, nl=3, shuffle_seed=3)
    Ar = rounded_matrix(M.hdg, FMT[precision])
    gs = BlockGS(Ar, vertex_patches(ts[-1], M.hdg.dpf))
    gs.inv = [stored_rows(np.linalg.inv(M.A[d, :][:, d].toarray()), FMT[precision]) for _, d in gs.patches]
    gs_exact = BlockGS(M.A, vertex_patches(ts[-1], M.hdg.dpf))
    rng = np.random.default_rng(3)
    for reverse in (False, True):
        g, u0 = rng.standard_normal((2, M.A.shape[0]))
        ud = dev(u0)
        hdg.hdg_smooth(ctx, -1, dev(g), ud, 1, reverse)
        uo = (gs.backward if reverse else gs.forward)(g, u0.copy())
        ue = (gs_exact.backward if reverse else gs_exact.forward)(g, u0.copy())
        assert rel(host(ud), uo) < 2e-5
        assert rel(uo, ue) > 20 * rel(host(ud), uo)


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("k,oseen", [(2, False), (3, False), (2, True)])
def test_precond_matches_rounded_model(precision, k, oseen):
    hdg = _hdg()
    ctx, F, M, fv, ts = case(k, precision, oseen=oseen, shuffle_seed=5)
    rng = np.random.default_rng(6)
    r = rng.standard_normal(M.A.shape[0])
    z_exact = M(r)
    Mr = round_hpmg(M, FMT[precision])
    z_model = Mr(r)
    z = host(hdg.hdg_precond_apply(ctx, dev(r)))
    assert rel(z, z_model) < 1e-4
    assert rel(z_model, z_exact) > 10 * rel(z, z_model)


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("k", [1, 3])
def test_solve_reaches_discrete_solution(precision, k):
    hdg = _hdg()
    ctx, F, M, fv, ts = case(k, precision, jitter=0.2, seed=4)
    oh = M.hdg
    ud, pd = oh.solve_direct(oh.load(fv))
    u, p, info = hdg.hdg_solve(ctx, F)
    eu, ep = relnorm(host(u), ud), relnorm(host(p), pd)
    print(f"16-bit precision {precision} k={k}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
    assert eu < 1e-8 and ep < 1e-8
    ctx32, F32, *_ = case(k, 1, jitter=0.2, seed=4)
    u32, p32, info32 = hdg.hdg_solve(ctx32, F32)
    # the 16-bit copies perturb the preconditioner, not the discrete problem
    assert info["krylov_its_total"] <= 1.5 * info32["krylov_its_total"] + 4


def _multi_case(k, precision, nrhs, **meshkw):
    from workloads import forcing_at_lattice
    from workloads.manufactured import fourier_forcing_2d
    hdg = _hdg()
    ms, ts, ps = hierarchy(2, 4, **meshkw)
    fine = ms[-1]
    fvs = [forcing_at_lattice(fine.coords, fine.cells, k, fourier_forcing_2d(j)) for j in range(nrhs)]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=1.0, gamma=100.0, precision=precision))
    F = torch.stack([hdg.hdg_load(ctx, dev(fv)) for fv in fvs])
    return ctx, F, ts, ps, fvs


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("nrhs,mesh", [(16, {}), (20, dict(shuffle_seed=9))])
def test_batched_tensor_core_precond_matches_model(precision, nrhs, mesh):
    """Batched preconditioner with the tensor-core order-k sweep (k = 3, 16 or 32 columns)
    against the CPU model of that sweep, column by column."""
    hdg = _hdg()
    k = 3
    ctx, F, ts, ps, fvs = _multi_case(k, precision, nrhs, **mesh)
    gen = torch.Generator(device=DEV).manual_seed(11)
    X = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    Z = host(hdg.hdg_precond_apply_multi(ctx, X))
    Xh = host(X)
    M = build_hpmg(ts, ps, k, 1.0, 1.0, 100.0)
    cols = (0, 1, nrhs - 1)
    exact = {r: M(Xh[r]) for r in cols}
    round_hpmg_tc(M, FMT[precision])
    for r in cols:
        zm = M(Xh[r])
        err = np.linalg.norm(Z[r] - zm) / np.linalg.norm(zm)
        gap = np.linalg.norm(zm - exact[r]) / np.linalg.norm(exact[r])
        # FP32 arithmetic on the device moves some values across a rounding boundary of
        # the 16-bit format (see test_batched_tensor_core_sweep_matches_model), and the
        # V-cycle's many sweeps carry those flips on: the device stays a fraction of the
        # rounding's own effect away from the model, where an unrounded (FP32) sweep
        # would sit at the full distance `gap`
        print(f"column {r}: device-model {err:.3e}, model-unrounded {gap:.3e}")
        assert err < 0.35 * gap


@pytest.mark.parametrize("nrhs", [16, 24])
def test_batched_tensor_core_solve_reaches_discrete_solution(nrhs):
    hdg = _hdg()
    k = 3
    ctx, F, ts, ps, fvs = _multi_case(k, hdg.HDG_MIXED_FP16, nrhs, jitter=0.2, seed=6)
    o = hdg.default_solve_opts()
    o.rtol, o.floor_rel, o.uzawa_tol = 1e-10, 1e-11, 1e-10
    U, P, infos = hdg.hdg_solve_multi(ctx, F, opts=o)
    ctx32, F32, *_ = _multi_case(k, hdg.HDG_MIXED_FP32, nrhs, jitter=0.2, seed=6)
    U32, P32, infos32 = hdg.hdg_solve_multi(ctx32, F32, opts=o)
    oh = HDG(ts[-1], k, nu=1.0, beta=1.0, gamma=100.0)
    for r in (0, nrhs - 1):
        ud, pd = oh.solve_direct(oh.load(fvs[r]))
        eu, ep = relnorm(host(U[r]), ud), relnorm(host(P[r]), pd)
        print(f"tensor-core batched column {r}: vs direct |du| {eu:.2e} |dp| {ep:.2e}")
        assert eu < 1e-8 and ep < 1e-8
    its = sum(i["krylov_its_total"] for i in infos)
    its32 = sum(i["krylov_its_total"] for i in infos32)
    assert its <= 1.5 * its32 + 4 * nrhs


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("mesh", [{}, dict(jitter=0.2, seed=2, shuffle_seed=4)])
def test_batched_tensor_core_sweep_matches_model(precision, mesh):
    """One order-k sweep (three colour phases) of the tensor-core kernel on 16 columns
    against the CPU model of the same sweep on the same inputs, forward and reverse.

    The device accumulates in FP32 where the model uses FP64, so now and then a value
    lands on the other side of a rounding boundary of the 16-bit format, and the later
    colour phases carry such flips on: a column either follows the model to FP32
    round-off or differs by a few such flips.  The test asks for most columns to follow
    the model far more closely than the unrounded sweep does, and for every column to
    stay well inside that distance."""
    hdg = _hdg()
    k, nrhs = 3, 16
    ctx, F, ts, ps, fvs = _multi_case(k, precision, nrhs, **mesh)
    M = build_hpmg(ts, ps, k, 1.0, 1.0, 100.0)
    gs_exact = BlockGS(M.A, vertex_patches(ts[-1], M.hdg.dpf))
    round_hpmg_tc(M, FMT[precision])
    rng = np.random.default_rng(21)
    G = rng.standard_normal((nrhs, M.A.shape[0]))
    U0 = rng.standard_normal((nrhs, M.A.shape[0]))
    ratios = []
    for reverse in (False, True):
        Ud = dev(U0)
        hdg.hdg_smooth_multi(ctx, -1, dev(G), Ud, 1, reverse)
        Ud = host(Ud)
        for r in range(nrhs):
            um = (M.gs.backward if reverse else M.gs.forward)(G[r], U0[r].copy())
            ue = (gs_exact.backward if reverse else gs_exact.forward)(G[r], U0[r].copy())
            err = np.linalg.norm(Ud[r] - um) / np.linalg.norm(um)
            gap = np.linalg.norm(um - ue) / np.linalg.norm(ue)
            ratios.append(err / gap)
    ratios = np.sort(ratios)
    print("device-model / model-unrounded per column:", " ".join(f"{x:.1e}" for x in ratios))
    # about 4e4 values are rounded per column and sweep here; an FP32 difference of 1e-7
    # relative flips a binary16 rounding (11 bits) with probability ~2e-4 and a bfloat16
    # one (8 bits) with ~3e-5, i.e. ~9 resp. ~1 flips per column, which puts the ratio
    # near sqrt(9 / 4e4) ~ 0.015 for binary16 and at 0 or a few 1e-3 for bfloat16
    assert np.median(ratios) < 0.06
    assert ratios[-1] < 0.3


@pytest.mark.parametrize("precision", [2, 3])
def test_batched_tensor_core_columns_are_independent(precision):
    """Each column's result depends on that column only (per-column scales, the columns as
    the M rows of the MMA tiles): permuting the 32 input columns permutes the sweep's and
    the preconditioner's output columns exactly."""
    hdg = _hdg()
    k, nrhs = 3, 32
    ctx, F, ts, ps, fvs = _multi_case(k, precision, nrhs, shuffle_seed=8)
    gen = torch.Generator(device=DEV).manual_seed(5)
    X = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    G = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    perm = torch.randperm(nrhs, generator=torch.Generator().manual_seed(3)).to(DEV)
    Z = host(hdg.hdg_precond_apply_multi(ctx, X))
    Zp = host(hdg.hdg_precond_apply_multi(ctx, X[perm].contiguous()))
    assert np.array_equal(Zp, Z[perm.cpu().numpy()])
    U = X.clone()
    hdg.hdg_smooth_multi(ctx, -1, G, U, 2, False)
    Up = X[perm].contiguous()
    hdg.hdg_smooth_multi(ctx, -1, G[perm].contiguous(), Up, 2, False)
    assert np.array_equal(host(Up), host(U)[perm.cpu().numpy()])


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_core_block_size_autotuned_and_bitwise_equal(precision):
    """The tensor-core sweep's block size (128 or 256 threads) is chosen by the autotuner
    (hdg_tune_batched reports 0 rows per thread and the block size) and does not change the
    result: both block sizes give bitwise the same preconditioner output."""
    hdg = _hdg()
    k, nrhs = 3, 32
    ctx, F, ts, ps, fvs = _multi_case(k, precision, nrhs)
    rb, nt, ms = hdg.hdg_tune_batched(ctx, nrhs)
    assert rb == 0 and nt in (128, 256) and ms > 0
    gen = torch.Generator(device=DEV).manual_seed(7)
    X = torch.randn(F.shape, dtype=torch.float64, device=DEV, generator=gen)
    outs = []
    for threads in (128, 256):
        hdg.hdg_set_batched_tile(ctx, 1, threads)
        outs.append(host(hdg.hdg_precond_apply_multi(ctx, X)))
    hdg.hdg_set_batched_tile(ctx, 0, 0)
    assert np.array_equal(outs[0], outs[1])
