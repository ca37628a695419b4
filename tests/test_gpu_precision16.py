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
from _util import hierarchy, forcing, rel
from _round16 import round_hpmg, stored_rows, rounded_matrix

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
    assert np.linalg.norm(host(u) - ud) < 1e-8 * np.linalg.norm(ud)
    assert np.linalg.norm(host(p) - pd) < 1e-6 * np.linalg.norm(pd)
    ctx32, F32, *_ = case(k, 1, jitter=0.2, seed=4)
    u32, p32, info32 = hdg.hdg_solve(ctx32, F32)
    # the 16-bit copies perturb the preconditioner, not the discrete problem
    assert info["krylov_its_total"] <= 1.5 * info32["krylov_its_total"] + 4
