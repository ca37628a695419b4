"""hdg_restrict_noalloc: the restriction for callers that cannot allocate device memory.

Called through the C ABI (ctypes, no Python wrapper logic) and compared with
hdg_restrict, the entry point that uses the context's own work buffers, on two
calls in a row (the shared fixed scratch array keeps the previous call's
contents, so the second call checks that nothing stale leaks through).  This
file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, ctx, level, rf, rc):
    s = torch.cuda.current_stream()
    return lib.hdg_restrict_noalloc(ctx.handle, level, ctypes.c_void_p(rf.data_ptr()),
                                    ctypes.c_void_p(rc.data_ptr()), ctypes.c_void_p(s.cuda_stream))


def test_restrict_noalloc_matches_restrict_twice():
    import paper_2303_06762_gb300 as hdg
    from workloads import unit_square_hierarchy
    lib = hdg.load_library()
    ms = unit_square_hierarchy(2, 4, jitter=0.2, seed=5)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=1, gamma=100.0, beta=1.0))
    s = ctx.sizes()
    rng = np.random.default_rng(0)
    for level in (3, 2, 1):
        nf, nc = int(s.n_dof_level[level]), int(s.n_dof_level[level - 1])
        for call in range(2):
            rf = torch.tensor(rng.standard_normal(nf), device="cuda:0")
            ref = hdg.hdg_restrict(ctx, level, rf)
            out = torch.full((nc,), np.nan, dtype=torch.float64, device="cuda:0")
            assert _call_noalloc(lib, ctx, level, rf, out) == 0
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (level, call)
    ctx.close()


def test_restrict_noalloc_rejects_oversized_level():
    import paper_2303_06762_gb300 as hdg
    from workloads import unit_square_hierarchy
    lib = hdg.load_library()
    ms = unit_square_hierarchy(2, 9)            # 2x2 .. 512x512; level 8's coarse mesh: 131072 cells
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=0, gamma=10.0))
    s = ctx.sizes()
    rf = torch.zeros(int(s.n_dof_level[8]), dtype=torch.float64, device="cuda:0")
    rc = torch.zeros(int(s.n_dof_level[7]), dtype=torch.float64, device="cuda:0")
    assert _call_noalloc(lib, ctx, 8, rf, rc) == 1       # HDG_ERR_INVALID_ARG
    assert b"more than the fixed scratch holds" in lib.hdg_last_error(ctx.handle)
    ctx.close()
