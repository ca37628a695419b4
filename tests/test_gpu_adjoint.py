"""GPU parity of per-cell viscosity, recovery of local fields, and the adjoint.

The adjoint gradients (forcing and per-cell viscosity) from hdg_adjoint are
compared with the oracle's adjoint (exact solves), itself pinned by finite
differences in tests/test_oracle_adjoint.py.  Tight solver tolerances make the
iterative GPU solves agree with the exact solves far below the comparison
tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
from workloads.manufactured import lattice_barycentric_2d
from oracle.hdg import HDG
from oracle.adjoint import objective_and_gradient
from _util import topo_of, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _case(k, beta=0.0, N0=2, nl=3, shuffle_seed=4):
    ms = unit_square_hierarchy(N0, nl, shuffle_seed=shuffle_seed)
    fine = ms[-1]
    t = topo_of(fine)
    rng = np.random.default_rng(7)
    nu = 1.0 * (1 + 0.1 * rng.uniform(-1, 1, fine.n_cells))
    fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(1.0, beta))
    ut = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().u) + \
        0.1 * rng.standard_normal(fv.shape)
    return ms, t, nu, fv, ut


def _tight(hdg):
    o = hdg.default_solve_opts()
    o.rtol, o.atol, o.floor_rel, o.uzawa_tol = 1e-12, 1e-14, 1e-12, 1e-11
    return o


def d(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("k", [1, 3])
def test_per_cell_viscosity_and_recovery(k):
    import paper_2303_06762_gb300 as hdg
    ms, t, nu, fv, ut = _case(k, beta=1.0)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=1.0, beta=1.0, gamma=100.0, nu_elem=d(nu))
    F = hdg.hdg_condense(ctx, prm, d(fv))
    oh = HDG(t, k, nu=1.0, beta=1.0, gamma=100.0, nu_elem=nu)
    A = hdg.hdg_get_element_matrices(ctx, -1).cpu().numpy()
    assert rel(A, np.stack([oh.element_matrix(c) for c in range(t.n_cells)])) < 1e-12
    assert rel(F.cpu().numpy(), oh.load(fv)) < 1e-12
    u, p, info = hdg.hdg_solve(ctx, F, opts=_tight(hdg))
    ud, pd = oh.solve_direct(oh.load(fv))
    assert rel(u.cpu().numpy(), ud) < 1e-9
    L, ul = hdg.hdg_recover(ctx, u, d(fv))
    L, ul = L.cpu().numpy(), ul.cpu().numpy()
    lam = lattice_barycentric_2d(k + 1)
    for c in range(0, t.n_cells, 7):
        coeffs = oh.recover_cell(c, ud, pd[c], fv[c])
        el = oh.cells[c].el
        _, uo, _, _ = oh.fields_at(c, coeffs, lam @ el.X)
        assert rel(ul[c], uo) < 1e-9
        # L_h is returned in an orthonormal P^k basis: ||L_h||_K^2 = |det J| sum of squares
        from oracle.quadrature import triangle_points
        xq, wq = triangle_points(el.X, k + 3)
        Lq, _, _, _ = oh.fields_at(c, coeffs, xq)
        norm_o = np.einsum("q,qij,qij->", wq, Lq, Lq)
        norm_g = 2 * el.area * np.sum(L[c] ** 2)
        assert abs(norm_g - norm_o) < 1e-9 * norm_o


@pytest.mark.parametrize("k,beta", [(1, 0.0), (2, 1.0)])
def test_adjoint_matches_oracle(k, beta):
    import paper_2303_06762_gb300 as hdg
    ms, t, nu, fv, ut = _case(k, beta=beta)
    Jo, gfo, gno, *_ = objective_and_gradient(t, k, fv, ut, nu, beta=beta)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=k, nu=1.0, beta=beta, gamma=100.0, nu_elem=d(nu))
    F = hdg.hdg_condense(ctx, prm, d(fv))
    o = _tight(hdg)
    u, p, _ = hdg.hdg_solve(ctx, F, opts=o)
    J, gf, gn, info = hdg.hdg_adjoint(ctx, d(fv), u, d(ut), opts=o)
    assert abs(J - Jo) < 1e-9 * Jo
    assert rel(gf.cpu().numpy(), gfo) < 1e-8
    assert rel(gn.cpu().numpy(), gno) < 1e-8
    assert info["krylov_its_total"] > 0


def test_autograd_function_and_mixed_precision_adjoint():
    import paper_2303_06762_gb300 as hdg
    from paper_2303_06762_gb300.autograd import StokesObjective
    k = 1
    ms, t, nu, fv, ut = _case(k)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    Jo, gfo, gno, *_ = objective_and_gradient(t, k, fv, ut, nu)
    f = d(fv).requires_grad_(True)
    n = d(nu).requires_grad_(True)
    prm = hdg.Params(k=k, nu=1.0, gamma=100.0, precision=hdg.HDG_MIXED_FP32)
    J = StokesObjective.apply(f, n, d(ut), ctx, prm, _tight(hdg))
    J.backward()
    assert abs(J.item() - Jo) < 1e-8 * Jo
    assert rel(f.grad.cpu().numpy(), gfo) < 1e-7
    assert rel(n.grad.cpu().numpy(), gno) < 1e-7
