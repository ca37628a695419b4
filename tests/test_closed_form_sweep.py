"""The closed-form patch update of the device sweeps, checked on the oracle's operator.

The block GS step u_P <- u_P + A_PP^-1 (g - A u)_P (Section 3.4.2) equals
A_PP^-1 (g_P - A_PE u_E), E the star cells' facets outside the patch, because A_PP is the
assembled patch matrix.  The FP64 kernels take that form directly.  The 2D FP32 kernels take it
with the augmented-Lagrangian term G_c d_c d_c^T (G_c = gamma nu / |K|) split off:

    u_P = A_PP^-1 (g_P - A0_PE u_E) - (A_PP^-1 D_P G) z,   z_c = d_{c,e} u_{e,0},

which needs (i) d_c to live on the first unknown of each facet, (ii) the patch rows to couple
outside the patch only through the facets of the star cells opposite the patch vertex (2D) or
the patch edge's end points (3D).  These tests build both forms cell by cell, as the kernels
do, and compare them with the step on the assembled operator.  The last test runs the three
forms of one sweep in FP32 (NumPy float32) and checks that the split form's error does not grow
with gamma, while the unsplit closed form's does.
"""
import numpy as np
import pytest

from oracle.hdg import HDG
from oracle.mg import vertex_patches
from _util import hierarchy


def _closed_steps(h, A, dofs, star_cells, outside, u, g):
    """The closed form and its AL split, assembled from the star cells' element matrices."""
    dpf = h.dpf
    P = np.linalg.inv(A[dofs][:, dofs].toarray())
    pos = {int(r): i for i, r in enumerate(dofs)}
    v = g[dofs].copy()
    v0 = g[dofs].copy()
    DG = np.zeros((len(dofs), len(star_cells)))
    z = np.zeros(len(star_cells))
    for s, c in enumerate(star_cells):
        Ac = h.element_matrix(c)
        A0c = h.element_matrix(c, with_al=False)
        d = h.cells[c].d
        G = h.eps_inv[c] / h.cells[c].area
        for fo in outside[s]:
            e_glob = h.l2g[c, fo * dpf:(fo + 1) * dpf]
            if e_glob[0] >= 0:
                z[s] += d[fo * dpf] * u[e_glob[0]]
        for f in range(Ac.shape[0] // dpf):
            if f in outside[s]:
                continue
            rows = h.l2g[c, f * dpf:(f + 1) * dpf]
            if rows[0] < 0:
                continue
            ip = [pos[int(r)] for r in rows]
            DG[ip[0], s] += G * d[f * dpf]
            for fo in outside[s]:
                e_glob = h.l2g[c, fo * dpf:(fo + 1) * dpf]
                if e_glob[0] >= 0:
                    v[ip] -= Ac[f * dpf:(f + 1) * dpf, fo * dpf:(fo + 1) * dpf] @ u[e_glob]
                    v0[ip] -= A0c[f * dpf:(f + 1) * dpf, fo * dpf:(fo + 1) * dpf] @ u[e_glob]
    return P @ v, P @ v0 - (P @ DG) @ z


@pytest.mark.parametrize("k,gamma", [(1, 1e2), (3, 1e4)])
def test_closed_form_and_al_split_2d(k, gamma):
    ms, ts, ps = hierarchy(4, 1, jitter=0.2, seed=3)
    t = ts[-1]
    h = HDG(t, k, nu=0.7, beta=1.0, gamma=gamma)
    A = h.matrix().tocsr()
    dpf = h.dpf
    for c in range(t.n_cells):
        d = h.cells[c].d
        # the oracle forms d by quadrature in physical coordinates: zero up to rounding
        assert np.abs(d[np.arange(d.size) % dpf != 0]).max() <= 1e-13 * np.abs(d).max()
    rng = np.random.default_rng(5)
    u, g = rng.standard_normal((2, A.shape[0]))
    for v, dofs in vertex_patches(t, dpf):
        star = [c for c in range(t.n_cells) if v in t.cells[c]]
        outside = [[list(t.cells[c]).index(v)] for c in star]   # facet f lies opposite vertex f
        ref = u[dofs] + np.linalg.inv(A[dofs][:, dofs].toarray()) @ (g[dofs] - A[dofs, :] @ u)
        closed, split = _closed_steps(h, A, dofs, star, outside, u, g)
        assert np.abs(closed - ref).max() <= 1e-9 * np.abs(ref).max()
        assert np.abs(split - ref).max() <= 1e-9 * np.abs(ref).max()


def test_closed_form_3d():
    from workloads.mesh3d import unit_cube
    from oracle.topology3d import build_topology_3d, edge_patches
    from oracle.hdg3d import HDG3D
    m = unit_cube(2, shuffle_seed=4)
    t = build_topology_3d(m.coords, m.cells)
    h = HDG3D(t, 1, nu=1.0, beta=1.0, gamma=1e4)
    A = h.matrix().tocsr()
    rng = np.random.default_rng(6)
    u, g = rng.standard_normal((2, A.shape[0]))
    for e, dofs in edge_patches(t, h.dpf):
        a, b = (int(x) for x in t.edges[e])
        star = [c for c in range(len(m.cells)) if a in m.cells[c] and b in m.cells[c]]
        outside = [[list(m.cells[c]).index(a), list(m.cells[c]).index(b)] for c in star]
        ref = u[dofs] + np.linalg.inv(A[dofs][:, dofs].toarray()) @ (g[dofs] - A[dofs, :] @ u)
        closed, split = _closed_steps(h, A, dofs, star, outside, u, g)
        assert np.abs(closed - ref).max() <= 1e-9 * np.abs(ref).max()
        assert np.abs(split - ref).max() <= 1e-9 * np.abs(ref).max()


def _fp32_sweep_errors(gamma):
    """One forward sweep from a random start in FP32 by the correction form, the closed form and
    the split closed form; residual error of each against the FP64 sweep, relative to the
    FP64 sweep's residual."""
    ms, ts, ps = hierarchy(6, 1)
    t = ts[-1]
    h = HDG(t, 1, nu=1.0, beta=1.0, gamma=gamma)
    A = h.matrix().tocsr()
    A0 = h.matrix(with_al=False).tocsr()
    AL = (A - A0).tocsr()
    n = A.shape[0]
    rng = np.random.default_rng(7)
    g, u0 = rng.standard_normal((2, n))
    ue = u0.copy()
    pats = []
    for _, d in vertex_patches(t, h.dpf):
        E = np.setdiff1d(np.arange(n), d)
        P = np.linalg.inv(A[d][:, d].toarray())
        ue[d] += P @ (g[d] - A[d, :] @ ue)
        pats.append((d, E, P.astype(np.float32), (P @ AL[d][:, E].toarray()).astype(np.float32),
                     A[d, :].astype(np.float32), A[d][:, E].astype(np.float32), A0[d][:, E].astype(np.float32)))
    out = {}
    for form in ("correction", "closed", "split"):
        u = u0.astype(np.float32)
        g32 = g.astype(np.float32)
        for d, E, P32, Q32, Ar, ApE, A0pE in pats:
            if form == "correction":
                u[d] = u[d] + P32 @ (g32[d] - Ar @ u)
            elif form == "closed":
                u[d] = P32 @ (g32[d] - ApE @ u[E])
            else:
                u[d] = P32 @ (g32[d] - A0pE @ u[E]) - Q32 @ u[E]
        du = u.astype(np.float64) - ue
        out[form] = np.linalg.norm(A @ du) / np.linalg.norm(g - A @ ue)
    return out


def test_split_removes_the_gamma_growth_of_fp32_rounding():
    lo, hi = _fp32_sweep_errors(1e2), _fp32_sweep_errors(1e5)
    assert hi["closed"] > 100 * lo["closed"]          # O(gamma) values meet the FP32 inverse
    assert hi["split"] < 10 * lo["split"]              # the split keeps them away
    assert hi["split"] < 1e-2 * hi["correction"]
