"""Block smoothers, intergrid transfer, h-multigrid and hp-multigrid (oracle).

TEST INFRASTRUCTURE ONLY.  Everything acts on assembled global sparse
matrices with plain sequential loops, in the order the paper states.

* Vertex patches (Section 3.4.2, subspaces V^{0,s}; Section 3.5 for order k):
  the patch of vertex s holds every unknown on the interior facets that
  contain s.  Patches are visited by colour of a proper vertex colouring,
  then by vertex id.
* Block Gauss–Seidel (Section 5: block GS for relaxation and smoothing):
  for each patch in turn u_s ← u_s + A_ss⁻¹ (g − A u)_s.  R^T, the transpose
  with respect to the skeleton inner product (eq. bjac and below), is the
  same sweep with the patches in reverse order.
* Damped block Jacobi (eq. bjac, the smoother of the theory): all patches
  against one residual, corrections summed and scaled by ς.
* Averaging transfer I_{l−1}^l (eq. avgOpt): evaluate Π^CR of the coarse
  function at each fine facet midpoint (inside a coarse cell: that cell's
  value; on a coarse facet: the mean of the two sides); fine boundary facets
  carry no unknowns.
* Harmonic-extension correction (eqs. div-transfer, harmonic-ex):
  𝓘 = (id − P^T) I with P^T the A^ε-orthogonal projection onto the fine
  unknowns on facets inside coarse cells.  Restriction = 𝓘ᵀ.
* Algorithm 1 (MG_h) with q = 1 (variable V-cycle, m(l−1) = growth·m(l)) or
  q = 2 (W-cycle), exact solve on the coarsest level.
* Oseen (Section 4.2: the same smoothers and transfers applied to A^{c,ε}):
  every lowest-order level carries its own convecting field, the RT_0 field
  whose facet fluxes are those of the finest field w_h (the mean of the two
  sides of each facet), summed over the two fine facets that make up each
  coarse facet (``lowest_order_convection``).  The coarsest solve is a dense
  LU factorisation instead of Cholesky.
* Algorithm 2 (MG_hp): m_p forward sweeps on A^ε_k, residual restricted by
  Π_k^0 (the transpose of the inclusion: the m = 0 normal and tangential
  coefficient of each facet), MG_h on the lowest-order operator of the same
  mesh, inclusion Π_0^k (injection of those coefficients), m_p reverse sweeps.
  Its additive form (Remark 3.4) sums the symmetric relaxation of g and the
  lowest-order correction of g.
"""

from __future__ import annotations

from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .cr import _bary
from .hdg import HDG
from .topology import Topology


def vertex_patches(topo: Topology, dpf: int):
    """Ordered list of (vertex, dof index array) for non-empty vertex patches."""
    inc = [[] for _ in range(topo.coords.shape[0])]
    for i, F in enumerate(topo.interior_facets):
        a, b = topo.facets[F]
        inc[a].append(i)
        inc[b].append(i)
    order = sorted(range(len(inc)), key=lambda v: (int(topo.vertex_colour[v]), v))
    out = []
    for v in order:
        if inc[v]:
            fac = sorted(inc[v])
            dofs = np.concatenate([np.arange(f * dpf, (f + 1) * dpf) for f in fac])
            out.append((v, dofs))
    return out


class BlockGS:
    """Sequential block Gauss–Seidel over vertex patches."""

    def __init__(self, A: sp.csr_matrix, patches):
        self.A = A.tocsr()
        self.patches = patches
        self.rows = [self.A[d, :] for _, d in patches]
        self.inv = [np.linalg.inv(self.A[d, :][:, d].toarray()) for _, d in patches]

    def forward(self, g, u):
        for (v, d), Ar, Ai in zip(self.patches, self.rows, self.inv):
            u[d] += Ai @ (g[d] - Ar @ u)
        return u

    def backward(self, g, u):
        for (v, d), Ar, Ai in zip(reversed(self.patches), reversed(self.rows), reversed(self.inv)):
            u[d] += Ai @ (g[d] - Ar @ u)
        return u


class BlockJacobi:
    """Damped block Jacobi over vertex patches, eq. bjac: every patch solves against the
    same residual and the corrections are summed, u ← u + ς Σ_s E_s A_ss⁻¹ E_sᵀ (g − A u).
    For symmetric A the operator is symmetric, so R^T = R (the forward and backward
    sweeps are the same step)."""

    def __init__(self, A: sp.csr_matrix, patches, damping: float = 0.5):
        self.A = A.tocsr()
        self.patches = patches
        self.damping = damping
        self.inv = [np.linalg.inv(self.A[d, :][:, d].toarray()) for _, d in patches]

    def forward(self, g, u):
        r = g - self.A @ u
        du = np.zeros_like(u)
        for (v, d), Ai in zip(self.patches, self.inv):
            du[d] += Ai @ r[d]
        u += self.damping * du
        return u

    backward = forward


def make_smoother(A: sp.csr_matrix, patches, smoother: str = "gs", damping: float = 0.5):
    """Block Gauss–Seidel (Section 5) or damped block Jacobi (eq. bjac) over `patches`."""
    if smoother == "gs":
        return BlockGS(A, patches)
    if smoother == "jacobi":
        return BlockJacobi(A, patches, damping)
    raise ValueError(smoother)


def averaging_prolongation(coarse: Topology, fine: Topology, parent: np.ndarray) -> sp.csr_matrix:
    """I_{l−1}^l of eq. avgOpt on lowest-order unknowns (2 per interior facet)."""
    rows, cols, vals = [], [], []

    def cr_weights(Kc, x):
        """Coefficients of Π^CR(v)(x) (2-vector) on coarse cell Kc w.r.t. coarse unknowns."""
        X = coarse.coords[coarse.cells[Kc]]
        lam = _bary(X, x[None, :])[0]
        out = []
        for i in range(3):
            psi = 1.0 - 2.0 * lam[i]
            F = coarse.cell_facets[Kc, i]
            ii = coarse.interior_index[F]
            if ii < 0:
                continue
            _, _, L, t, nF = coarse.facet_geometry(F)
            out.append((2 * ii, psi * nF / np.sqrt(L)))
            out.append((2 * ii + 1, psi * t / np.sqrt(L)))
        return out

    for i, F in enumerate(fine.interior_facets):
        c0, c1 = fine.facet_cells[F]
        xl, xh, L, t, nF = fine.facet_geometry(F)
        mid = 0.5 * (xl + xh)
        p0, p1 = parent[c0], parent[c1]
        sides = [p0] if p0 == p1 else [p0, p1]
        w = 1.0 / len(sides)
        for Kc in sides:
            for col, vec in cr_weights(Kc, mid):
                rows += [2 * i, 2 * i + 1]
                cols += [col, col]
                vals += [w * np.sqrt(L) * (vec @ nF), w * np.sqrt(L) * (vec @ t)]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * fine.n_interior, 2 * coarse.n_interior))


def interior_fine_dofs(fine: Topology, parent: np.ndarray) -> np.ndarray:
    """Lowest-order unknowns on fine facets inside coarse cells (the set T)."""
    out = []
    for i, F in enumerate(fine.interior_facets):
        c0, c1 = fine.facet_cells[F]
        if parent[c0] == parent[c1]:
            out += [2 * i, 2 * i + 1]
    return np.asarray(out, dtype=np.int64)


def harmonic_prolongation(A_fine: sp.csr_matrix, I_avg: sp.csr_matrix, T: np.ndarray) -> sp.csr_matrix:
    """𝓘 = (id − P^T) I: replace the T-part by the discrete A^ε-harmonic extension."""
    A = A_fine.tocsr()
    ATT = A[T, :][:, T].tocsc()
    AI = (A @ I_avg).tocsr()[T, :]
    corr = (spla.inv(ATT) @ AI).tocoo()
    ET = sp.csr_matrix((np.ones(len(T)), (T, np.arange(len(T)))), shape=(A.shape[0], len(T)))
    return (I_avg - ET @ corr).tocsr()


class Level:
    def __init__(self, hdg: HDG, smoother: str = "gs", damping: float = 0.5):
        self.hdg = hdg
        self.A = hdg.matrix(with_al=True).tocsr()
        # the level's smoother (named gs for block GS, the default; damped block Jacobi otherwise)
        self.gs = make_smoother(self.A, vertex_patches(hdg.topo, hdg.dpf), smoother, damping)
        self.P: Optional[sp.csr_matrix] = None    # prolongation from the level below


class MGh:
    """Algorithm 1 on lowest-order levels 1..J (index 0 = coarsest)."""

    def __init__(self, levels: List[Level], parents: List[np.ndarray], growth: int = 2,
                 symmetric: bool = True):
        self.levels = levels
        self.growth = growth
        for l in range(1, len(levels)):
            Ia = averaging_prolongation(levels[l - 1].hdg.topo, levels[l].hdg.topo, parents[l])
            T = interior_fine_dofs(levels[l].hdg.topo, parents[l])
            levels[l].P = harmonic_prolongation(levels[l].A, Ia, T)
        A0 = levels[0].A.toarray()
        self.symmetric = symmetric
        self.coarse = sla.cho_factor(A0) if symmetric else sla.lu_factor(A0)

    def cycle(self, l: int, g, u0, m: int, q: int = 1):
        if l == 0:
            if self.symmetric:
                return sla.cho_solve(self.coarse, g)
            return sla.lu_solve(self.coarse, g)
        L = self.levels[l]
        u = u0.copy()
        for _ in range(m):
            L.gs.forward(g, u)
        r = L.P.T @ (g - L.A @ u)
        du = np.zeros(r.shape[0])
        for _ in range(q):
            du = self.cycle(l - 1, r, du, m * self.growth if q == 1 else m, q)
        u += L.P @ du
        for _ in range(m):
            L.gs.backward(g, u)
        return u

    def __call__(self, g, m: int, q: int = 1, u0=None):
        J = len(self.levels) - 1
        return self.cycle(J, g, np.zeros_like(g) if u0 is None else u0, m, q)


def inclusion_matrix(n_int: int, k: int) -> sp.csr_matrix:
    """Π_0^k: lowest-order facet unknowns -> order-k unknowns (injection)."""
    dpf = 2 * (k + 1)
    rows, cols = [], []
    for i in range(n_int):
        rows += [i * dpf, i * dpf + (k + 1)]
        cols += [2 * i, 2 * i + 1]
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n_int * dpf, 2 * n_int))


class MGhp:
    """Algorithm 2: z = MG_hp(g, 0, m_p, m_h, q).

    additive=True gives the additive form of the same space decomposition (Remark 3.4,
    eq. hpSubspace): the relaxation part (m_p forward then m_p backward sweeps from zero)
    and the lowest-order correction Π_0^k MG_h(Π_k^0 g) are both computed from g and
    summed, z = R_sym g + Π_0^k MG_h(Π_k^0 g)."""

    def __init__(self, hdg_k: HDG, mgh: MGh, m_p: int = 1, m_h: int = 1, q: int = 1,
                 smoother: str = "gs", damping: float = 0.5, additive: bool = False):
        self.hdg = hdg_k
        self.A = hdg_k.matrix(with_al=True).tocsr()
        self.k = hdg_k.k
        self.mgh = mgh
        self.m_p, self.m_h, self.q = m_p, m_h, q
        self.additive = additive
        if self.k > 0:
            self.gs = make_smoother(self.A, vertex_patches(hdg_k.topo, hdg_k.dpf), smoother, damping)
            self.Pi = inclusion_matrix(hdg_k.topo.n_interior, self.k)

    def __call__(self, g, u0=None):
        if self.k == 0:
            return self.mgh(g, self.m_h, self.q, u0)
        if self.additive:
            z = np.zeros_like(g)
            for _ in range(self.m_p):
                self.gs.forward(g, z)
            for _ in range(self.m_p):
                self.gs.backward(g, z)
            return z + self.Pi @ self.mgh(self.Pi.T @ g, self.m_h, self.q)
        u = np.zeros_like(g) if u0 is None else u0.copy()
        for _ in range(self.m_p):
            self.gs.forward(g, u)
        r0 = self.Pi.T @ (g - self.A @ u)
        du = self.mgh(r0, self.m_h, self.q)
        u += self.Pi @ du
        for _ in range(self.m_p):
            self.gs.backward(g, u)
        return u


def _outward_normal(X: np.ndarray, f: int):
    a, b = [v for v in range(3) if v != f]
    t = X[b] - X[a]
    L = float(np.hypot(t[0], t[1]))
    n = np.array([t[1], -t[0]]) / L
    if n @ (0.5 * (X[a] + X[b]) - X[f]) < 0:
        n = -n
    return a, b, L, n


def _lattice_values_at(q: int, vals: np.ndarray, lam_pts: np.ndarray) -> np.ndarray:
    """Evaluate the degree-q polynomial with lattice values `vals` (n_lat, 2) at
    points given by barycentric coordinates lam_pts (m, 3)."""
    from workloads.manufactured import lattice_barycentric_2d
    lat = lattice_barycentric_2d(q)
    ex = [(d - b, b) for d in range(q + 1) for b in range(d + 1)]

    def V(lam):
        return np.stack([lam[:, 1] ** a * lam[:, 2] ** b for a, b in ex], axis=1)
    return V(lam_pts) @ np.linalg.solve(V(lat), vals)


def lowest_order_convection(topos: List[Topology], parents: List[np.ndarray],
                            conv: np.ndarray) -> List[np.ndarray]:
    """Convecting field of every lowest-order level, (n_cells_l, 3, 2) values at
    the cell vertices (the degree-1 lattice), index 0 = coarsest.

    Reading of Section 4.2 for the coarse operators A^{c,ε}_{0,l}: on the finest
    mesh the field is the RT_0 function with the facet fluxes ∫_F w_h·n of the
    given order-k field (mean of the two adjacent cells), and on each coarser
    mesh the RT_0 function whose flux through a coarse facet is the sum of the
    fluxes through its two fine halves.  Divergence-free, normal-continuous
    fields with w·n = 0 on ∂Ω stay so on every level.
    """
    J = len(topos) - 1
    conv = np.asarray(conv, dtype=float)
    q = 0
    while (q + 1) * (q + 2) // 2 < conv.shape[1]:
        q += 1
    s_gl, w_gl = np.polynomial.legendre.leggauss(q + 2)
    s_gl, w_gl = 0.5 * (s_gl + 1.0), 0.5 * w_gl
    fine = topos[J]
    flux = np.zeros((fine.n_cells, 3))            # outward flux per (cell, local facet)
    for c in range(fine.n_cells):
        X = fine.coords[fine.cells[c]]
        for f in range(3):
            a, b, L, n = _outward_normal(X, f)
            lam = np.zeros((len(s_gl), 3))
            lam[:, a] = 1.0 - s_gl
            lam[:, b] = s_gl
            w = _lattice_values_at(q, conv[c], lam)
            flux[c, f] = L * (w_gl @ (w @ n))
    for F in fine.interior_facets:
        c0, c1 = fine.facet_cells[F]
        f0 = int(np.where(fine.cell_facets[c0] == F)[0][0])
        f1 = int(np.where(fine.cell_facets[c1] == F)[0][0])
        v = 0.5 * (flux[c0, f0] - flux[c1, f1])
        flux[c0, f0], flux[c1, f1] = v, -v
    fluxes = [None] * (J + 1)
    fluxes[J] = flux
    for l in range(J, 0, -1):
        tf, tc = topos[l], topos[l - 1]
        fc = np.zeros((tc.n_cells, 3))
        for c in range(tf.n_cells):
            P = int(parents[l][c])
            Xc = tc.coords[tc.cells[P]]
            for lf in range(3):
                F = tf.cell_facets[c, lf]
                o = tf.facet_cells[F]
                if o[1] >= 0 and parents[l][o[0]] == parents[l][o[1]]:
                    continue                      # facet inside the coarse cell
                lo, hi = tf.facets[F]
                mid = 0.5 * (tf.coords[lo] + tf.coords[hi])
                lamc = _bary_point(Xc, mid)
                fc[P, int(np.argmin(np.abs(lamc)))] += fluxes[l][c, lf]
        fluxes[l - 1] = fc
    out = []
    for l in range(J + 1):
        t = topos[l]
        vals = np.zeros((t.n_cells, 3, 2))
        for c in range(t.n_cells):
            X = t.coords[t.cells[c]]
            area = t.cell_area(c)
            for v in range(3):
                for f in range(3):
                    if f != v:
                        vals[c, v] += fluxes[l][c, f] * (X[v] - X[f]) / (2.0 * area)
        out.append(vals)
    return out


def _bary_point(X: np.ndarray, x: np.ndarray) -> np.ndarray:
    T = np.array([[X[0, 0], X[1, 0], X[2, 0]], [X[0, 1], X[1, 1], X[2, 1]], [1.0, 1.0, 1.0]])
    return np.linalg.solve(T, np.array([x[0], x[1], 1.0]))


def build_hpmg(topos: List[Topology], parents: List[np.ndarray], k: int, nu: float, beta: float,
               gamma: float, m_p: int = 1, m_h: int = 1, q: int = 1, growth: int = 2,
               hdg_k: Optional[HDG] = None, conv: Optional[np.ndarray] = None,
               conv_transpose: bool = False, smoother: str = "gs", damping: float = 0.5,
               additive: bool = False) -> MGhp:
    """hp-multigrid on the hierarchy topos[0] (coarsest) .. topos[-1] (finest).

    conv: lattice values (n_cells_fine, n_lat(k+1), 2) of the convecting field
    on the finest mesh (Oseen), or None (generalized Stokes).  smoother: "gs" (block
    Gauss–Seidel, Section 5) or "jacobi" (damped block Jacobi of eq. bjac with
    ς = damping) on every level; additive: the additive form of Algorithm 2 (MGhp).
    """
    conv_l = [None] * len(topos) if conv is None else lowest_order_convection(topos, parents, conv)
    levels = [Level(HDG(t, 0, nu=nu, beta=beta, gamma=gamma, conv=cl, conv_transpose=conv_transpose),
                    smoother, damping)
              for t, cl in zip(topos, conv_l)]
    mgh = MGh(levels, parents, growth=growth, symmetric=conv is None)
    if hdg_k is None:
        hdg_k = HDG(topos[-1], k, nu=nu, beta=beta, gamma=gamma, conv=conv,
                    conv_transpose=conv_transpose)
    return MGhp(hdg_k, mgh, m_p=m_p, m_h=m_h, q=q, smoother=smoother, damping=damping, additive=additive)
