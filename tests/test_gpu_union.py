"""Several uneven meshes in one solve: the disjoint union of their hierarchies (one context, one
captured preconditioner graph, every kernel launch covering all meshes) solves the block-diagonal
system of all meshes; each mesh's block matches its own exact discrete solution (the oracle's
direct solve) and the library's single-mesh solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
from workloads.mesh2d import disjoint_union
from oracle.hdg import HDG
from _util import topo_of, relnorm, parity_opts

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("precision", [0, 1])
def test_union_solve_matches_each_mesh(precision):
    import paper_2303_06762_gb300 as hdg
    k = 2
    hs = [unit_square_hierarchy(N0, 3) for N0 in (2, 3, 5)]          # N = 8, 12, 20
    u_h = disjoint_union(hs)
    sol = curl_bubble_2d()
    fvs = [forcing_at_lattice(h[-1].coords, h[-1].cells, k, sol.forcing(1.0, 1.0)) for h in hs]
    ctx = hdg.hdg_setup_mesh_hierarchy(u_h)
    F = hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=1.0, gamma=100.0, precision=precision),
                         torch.tensor(np.concatenate(fvs), device=DEV))
    opts = parity_opts(hdg, 100.0) if precision == 0 else hdg.default_solve_opts()
    u, p, info = hdg.hdg_solve(ctx, F, opts=opts)
    u, p = u.cpu().numpy(), p.cpu().numpy()
    for h, fv, (su, sp) in zip(hs, fvs, hdg.union_slices(hs, k)):
        oh = HDG(topo_of(h[-1]), k, nu=1.0, beta=1.0, gamma=100.0)
        ud, pd = oh.solve_direct(oh.load(fv))
        eu, ep = relnorm(u[su], ud), relnorm(p[sp], pd)
        print(f"union, precision {precision}, N={h[-1].N}: |du| {eu:.2e} |dp| {ep:.2e}")
        assert eu < (1e-10 if precision == 0 else 1e-8) and ep < (1e-9 if precision == 0 else 1e-8)
    ctx.close()
