"""GPU parity of the Picard iteration for steady Navier-Stokes (hdg_picard)
against the oracle's Picard iteration with exact solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import curl_bubble_2d, forcing_at_lattice
from oracle.navier_stokes import picard
from _util import hierarchy, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SOL = curl_bubble_2d()


@pytest.mark.parametrize("k,Re,precision", [(1, 1.0, 0), (2, 10.0, 1)])
def test_picard_matches_oracle(k, Re, precision):
    import paper_2303_06762_gb300 as hdg
    nu = 1.0 / Re
    ms, ts, ps = hierarchy(2, 3, shuffle_seed=2)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, SOL.forcing(nu, 0.0, conv=SOL.u))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=100.0, precision=precision)
    u, p, steps, dist = hdg.hdg_picard(ctx, prm, torch.tensor(fv, device=DEV), tol=1e-9, max_steps=40, opts=o)
    uo, po, n, do, h, w = picard(ts[-1], k, fv, nu, gamma=100.0, tol=1e-9)
    assert steps == n
    assert dist < 1e-9
    assert rel(u.cpu().numpy(), uo) < 1e-8
    pm = p.cpu().numpy()
    pm = pm - (h.area @ pm) / h.area.sum()
    pom = po - (h.area @ po) / h.area.sum()
    assert rel(pm, pom) < 1e-7
