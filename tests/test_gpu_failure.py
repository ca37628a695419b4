"""Failure detection on the GPU without a fault: the bounded waits of the bulk-copy
order-k sweep.

The limit of the first wait is set to zero through hdg_set_wait_limit, so every thread
block of the sweep records a timeout, waits (bounded) for its copies to land and skips
its update.  The entry points must report HDG_ERR_TIMEOUT, clear the flag, and leave the
context usable: with the default limit restored the same context solves to the exact
discrete solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d
from oracle.hdg import HDG
from _util import hierarchy, forcing

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_bulk_copy_wait_timeout_is_reported_and_context_stays_usable():
    import paper_2303_06762_gb300 as hdg
    k = 3
    ms, ts, ps = hierarchy(2, 3)
    fv = forcing(ms[-1], k, curl_bubble_2d(), 1.0, 1.0)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    F = hdg.hdg_condense(ctx, hdg.Params(k=k, beta=1.0, gamma=100.0, precision=hdg.HDG_MIXED_FP32),
                         torch.tensor(fv, device=DEV))
    hdg.hdg_set_wait_limit(ctx, 0)
    o = hdg.default_solve_opts()
    o.max_it = 3
    o.max_uzawa = 1
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_solve(ctx, F, opts=o)
    assert e.value.status == 10 and "timed out" in str(e.value)
    r = torch.randn(ctx.sizes().n_dof, dtype=torch.float64, device=DEV)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_precond_apply(ctx, r)
    assert e.value.status == 10
    u = torch.zeros_like(r)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_smooth(ctx, -1, r, u, 1, False)
    assert e.value.status == 10
    # the flag was cleared by each report; with the default limit the context works again
    hdg.hdg_set_wait_limit(ctx, 1_000_000_000)
    z = hdg.hdg_precond_apply(ctx, r)
    assert torch.isfinite(z).all()
    u, p, info = hdg.hdg_solve(ctx, F)
    oh = HDG(ts[-1], k, gamma=100.0, beta=1.0)
    ud, pd = oh.solve_direct(oh.load(fv))
    torch.cuda.synchronize()
    assert np.linalg.norm(u.cpu().numpy() - ud) < 1e-8 * np.linalg.norm(ud)
    with pytest.raises(hdg.HdgError) as e:
        hdg.hdg_set_wait_limit(ctx, -1)
    assert e.value.status == 1
    ctx.close()
