"""Oracle pins of the solver variants: the damped block-Jacobi smoother (eq. bjac), the
additive form of Algorithm 2 (Remark 3.4) and the preconditioned conjugate gradients of
Section 5 (the paper's Krylov method for the generalized Stokes problem)."""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import curl_bubble_2d
from oracle.hdg import HDG
from oracle.mg import BlockGS, BlockJacobi, build_hpmg, vertex_patches
from oracle.krylov import pcg, uzawa
from _util import hierarchy, forcing, relnorm


def _level(nl=3, k=1, gamma=100.0, **kw):
    ms, ts, ps = hierarchy(2, nl, **kw)
    h = HDG(ts[-1], k, beta=1.0, gamma=gamma)
    return ms, ts, ps, h


def test_jacobi_on_one_colour_is_that_gauss_seidel_phase():
    """Patches of one colour share no cell, hence no matrix entry: the undamped block
    Jacobi step over them is exactly the block GS phase of that colour."""
    ms, ts, ps, h = _level(shuffle_seed=2)
    A = h.matrix()
    pats = vertex_patches(h.topo, h.dpf)
    col = h.topo.vertex_colour
    rng = np.random.default_rng(0)
    for c in np.unique(col):
        sub = [(v, d) for v, d in pats if col[v] == c]
        g, u = rng.standard_normal((2, A.shape[0]))
        a = BlockGS(A, sub).forward(g, u.copy())
        b = BlockJacobi(A, sub, damping=1.0).forward(g, u.copy())
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_jacobi_symmetric_and_colour_bounded():
    """R = s sum_s E_s A_ss^-1 E_s^T is symmetric, and the eigenvalues of R A lie in
    (0, s n_c] with n_c the number of colours (each colour's patch projections are
    A-orthogonal, so their sum is a projection): s = 1/2 with 3 colours contracts."""
    ms, ts, ps, h = _level(nl=2, k=1, gamma=1e4, jitter=0.2, seed=3)
    A = h.matrix().toarray()
    J = BlockJacobi(sp.csr_matrix(A), vertex_patches(h.topo, h.dpf), damping=0.5)
    n = A.shape[0]
    R = np.stack([J.forward(e, np.zeros(n)) for e in np.eye(n)], axis=1)
    assert np.abs(R - R.T).max() <= 1e-12 * np.abs(R).max()
    lam = np.linalg.eigvals(R @ A).real
    nc = len(np.unique(h.topo.vertex_colour))
    assert lam.min() > 0 and lam.max() <= 0.5 * nc * (1 + 1e-10)
    assert np.abs(1 - lam).max() < 1


@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_additive_hpmg_symmetric_positive_definite(smoother):
    ms, ts, ps, h = _level(nl=3, k=2)
    M = build_hpmg(ts, ps, 2, 1.0, 1.0, 100.0, hdg_k=h, smoother=smoother, additive=True)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal((2, M.A.shape[0]))
    assert abs(x @ M(y) - M(x) @ y) <= 1e-11 * abs(x @ M(y))
    assert x @ M(x) > 0


def test_additive_degrades_with_gamma_and_k():
    """Remark 3.4: the additive form needs many more iterations than Algorithm 2, and
    more so as eps -> 0 and k grows."""
    ms, ts, ps = hierarchy(2, 3)

    def its(k, gamma, additive):
        h = HDG(ts[-1], k, beta=1.0, gamma=gamma)
        M = build_hpmg(ts, ps, k, 1.0, 1.0, gamma, hdg_k=h, additive=additive)
        F = h.load(forcing(ms[-1], k, curl_bubble_2d(), 1.0, 1.0))
        return pcg(M.A, F, np.zeros_like(F), M)[1]

    for k in (1, 3):
        mult = [its(k, g, False) for g in (1.0, 1e4)]
        add = [its(k, g, True) for g in (1.0, 1e4)]
        assert add[0] >= 3 * mult[0] and add[1] >= 3 * mult[1]
        assert add[1] - add[0] > mult[1] - mult[0]
    assert its(3, 1e4, True) > its(1, 1e4, True)


def test_pcg_finite_termination_and_exact_preconditioner():
    """CG on an SPD matrix with three distinct eigenvalues terminates in three steps;
    with the exact inverse as preconditioner in one."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Q @ np.diag(np.repeat([1.0, 4.0, 9.0], 4)) @ Q.T
    b = rng.standard_normal(12)
    x, its, rn, _ = pcg(A, b, np.zeros(12), lambda r: r, rtol=1e-12, atol=0.0)
    assert its == 3 and relnorm(x, np.linalg.solve(A, b)) < 1e-12
    Ainv = np.linalg.inv(A)
    x, its, rn, _ = pcg(A, b, np.zeros(12), lambda r: Ainv @ r, rtol=1e-12, atol=0.0)
    assert its == 1 and relnorm(x, np.linalg.solve(A, b)) < 1e-12


@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_uzawa_with_pcg_reaches_discrete_solution(smoother):
    ms, ts, ps, h = _level(nl=3, k=2)
    M = build_hpmg(ts, ps, 2, 1.0, 1.0, 100.0, hdg_k=h, smoother=smoother)
    F = h.load(forcing(ms[-1], 2, curl_bubble_2d(), 1.0, 1.0))
    r = uzawa(M.A, h.flux_matrix(), h.area, h.eps_inv, F, M, krylov="pcg")
    u, p = h.solve_direct(F)
    assert relnorm(r.u, u) < 1e-8 and relnorm(r.p, p) < 1e-8
    assert r.div_l2 < 1e-9           # div u_h = eps dp: at the Uzawa tolerance
