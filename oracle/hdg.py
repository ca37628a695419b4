"""H(div)-HDG local systems, static condensation and the exact discrete solution.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Scheme (Section 3.2, eq. stWeak): find (L_h, u_h, û_h, p_h) in
W^k × RT_k × V̂^k × W^k with, on every cell,
  (ν⁻¹L, G) + (∇u, G) − ⟨tng(u − û), G n⟩                      = 0,
  −(L, ∇v) + ⟨L n, tng(v − v̂)⟩ + β(u, v) − (p, div v)           = (f, v),
  (div u, q)                                                        = 0.
The oracle writes this full local matrix over (L, u, û, p) by quadrature in
physical coordinates, then eliminates the local unknowns (L, the interior RT
moments, the mean-free part of p) by a plain dense Schur complement
(Section 3.2, "we first eliminate the local variables").  What remains per
cell is the condensed matrix A_K on the 3(2k+2) facet unknowns (RT normal
moments and tangential Legendre coefficients), the condensed load F_K, and
the flux row d_K (∫_{∂K} v·n of each unknown) that carries B (eq. stOptForm).
The augmented-Lagrangian operator adds ε⁻¹|K|⁻¹ d_K d_Kᵀ with ε⁻¹ = γν
(eq. stALform, written per cell because (div u, div v)_K = |K|⁻¹(d_K·u)(d_K·v)
for the piecewise-constant divergence of the global space).

Local unknown order on a cell (the layout the library uses as well): facet
f = 0, 1, 2 (opposite local vertex f), and within a facet the normal moments
m = 0..k followed by the tangential coefficients m = 0..k.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from workloads.manufactured import lattice_barycentric_2d

from .quadrature import triangle_points
from .spaces import Element, exponents
from .topology import Topology


def _signature(X, gv, k, nu, beta, conv=None, conv_t=False):
    rel = np.ascontiguousarray(X - X[0])
    ranks = tuple(np.argsort(np.argsort(np.asarray(gv))).tolist())
    cb = None if conv is None else np.ascontiguousarray(conv, dtype=float).tobytes()
    return (rel.tobytes(), ranks, k, float(nu), float(beta), cb, bool(conv_t))


def lattice_degree(n_lat: int) -> int:
    q = 0
    while (q + 1) * (q + 2) // 2 < n_lat:
        q += 1
    assert (q + 1) * (q + 2) // 2 == n_lat, "not a triangle lattice size"
    return q


# relative threshold below which w·n counts as zero in the frozen Newton switch
NEWTON_TIE = 1e-10


def upwind_facet_points(k: int, q_w: int) -> int:
    """Gauss–Legendre points per facet for the upwind terms: exact for degree q_w + 2k + 2."""
    return (q_w + 2 * k + 4) // 2


@dataclass
class CondensedCell:
    A: np.ndarray        # (ng, ng) condensed matrix without the AL term
    d: np.ndarray        # (ng,) flux row: d·x = ∫_{∂K} u·n_K
    Fmap: np.ndarray     # (ng, n_lat*2) lattice forcing -> condensed load
    area: float
    # recovery: local unknowns y_l = Rf f - Rg x_g - Rp p_K
    Rf: np.ndarray
    Rg: np.ndarray
    Rp: np.ndarray
    el: Element
    lat_inv: np.ndarray  # lattice Vandermonde inverse (monomials of degree k+1)
    Fextra: Optional[np.ndarray] = None   # condensed fixed load (Newton), (ng,)
    Rextra: Optional[np.ndarray] = None   # its contribution to the local unknowns


def local_system(el: Element, nu: float, beta: float, conv=None, conv_transpose: bool = False,
                 newton_uhat=None, newton_boundary=(False, False, False)):
    """Full local matrix over (L, u, û, p), forcing map and index sets.

    conv: optional lattice values (n_lat_w, 2) of the convecting field w_h on
    this cell (degree q_w lattice, same ordering as the forcing).  It adds the
    upwind form of Section 4.1 with the Picard field w_h (eq. nsWeak):
      -(u, (w·∇)v)_K + <(w·n)^+ tng u + (w·n)^- tng û, tng(v - v̂)>_{∂K},
    i.e. u^up takes the trace of u where w·n_K > 0 and of û where w·n_K < 0,
    switched pointwise at the Gauss points of upwind_facet_points(k, q_w).
    conv_transpose: use the transpose of that (u, û) block instead.  Because
    the remaining blocks satisfy Mᵀ = S M S with S = diag(-I_L, I_u, I_û, -I_p),
    the local system with the transposed convection block is S Mᵀ S: the
    system whose solution gives the adjoint (Section 4.1 with A10's objective).
    newton_uhat: with conv = u_old (the previous velocity at the lattice), the
    (3, k+1) facet coefficients of the previous û_old on this cell's facets.
    It adds the Newton term of Section 4.2, C_h(δu; u_old, v): the derivative of
    the upwind form in its convecting argument with the switch frozen at
    u_old·n_K, i.e. -(u_old, (δu·∇)v) + <(δu·n_K) u_old^up, tng(v - v̂)> with
    u_old^up = tng u_old where u_old·n_K > NEWTON_TIE·max|w| (the lattice values)
    and tng û_old elsewhere and on the facets flagged in newton_boundary
    (Dirichlet facets).  The
    unknowns are then the new iterate itself: the right-hand side gains
    C_h(u_old; u_old, v), returned as info["rhs_extra"].
    """
    k = el.k
    npk = len(exponents(k))
    nL, nrt, nh, npp = 4 * npk, el.n_rt, 3 * (k + 1), npk
    oL, ou, oh, op = 0, nL, nL + nrt, nL + nrt + nh
    n = op + npp
    M = np.zeros((n, n))
    xq, wq = triangle_points(el.X, k + 3 if conv is None else k + 4)
    Pk = el.mono(xq, k)
    mean = (wq @ Pk) / el.area
    pv = Pk - mean[None, :]
    pv[:, 0] = 1.0                      # exponents(k)[0] == (0, 0): global P0 part
    U = el.rt_values(xq)
    GU = el.rt_grads(xq)
    DU = GU[:, :, 0, 0] + GU[:, :, 1, 1]
    Mp = (Pk * wq[:, None]).T @ Pk
    for ce in range(4):
        M[oL + ce * npk:oL + (ce + 1) * npk, oL + ce * npk:oL + (ce + 1) * npk] = Mp / nu
    # (∇u, G)
    for c in range(2):
        for e in range(2):
            ce = 2 * c + e
            M[oL + ce * npk:oL + (ce + 1) * npk, ou:ou + nrt] += (Pk * wq[:, None]).T @ GU[:, :, c, e]
    for f in range(3):
        fd = el.facets[f]
        s, xf, wf = el.facet_points(f, k + 3)
        Uf = el.rt_values(xf)
        nK = fd["nK"]
        tngU = Uf - np.einsum("qi,c->qic", Uf @ nK, nK)
        Pf = el.mono(xf, k)
        lm = el.facet_legendre(f, s)
        for c in range(2):
            for e in range(2):
                ce = 2 * c + e
                rows = slice(oL + ce * npk, oL + (ce + 1) * npk)
                # − ⟨tng(u), G n⟩
                M[rows, ou:ou + nrt] -= (Pf * (wf * nK[e])[:, None]).T @ tngU[:, :, c]
                # + ⟨tng(û), G n⟩ with û = ℓ_m t_F on this facet
                M[rows, oh + f * (k + 1):oh + (f + 1) * (k + 1)] += \
                    (Pf * (wf * nK[e] * fd["t"][c])[:, None]).T @ lm
    # −(L, ∇v) + ⟨L n, tng(v)⟩ and −⟨L n, tng(v̂)⟩ are the negative transposes
    M[ou:ou + nrt, oL:oL + nL] = -M[oL:oL + nL, ou:ou + nrt].T
    M[oh:oh + nh, oL:oL + nL] = -M[oL:oL + nL, oh:oh + nh].T
    M[ou:ou + nrt, ou:ou + nrt] += beta * np.einsum("q,qic,qjc->ij", wq, U, U)
    Bd = np.einsum("q,qi,qj->ij", wq, DU, pv)
    M[ou:ou + nrt, op:op + npp] = -Bd
    M[op:op + npp, ou:ou + nrt] = Bd.T
    if conv is not None:
        conv = np.asarray(conv, dtype=float)
        q_w = lattice_degree(conv.shape[0])
        lam_w = lattice_barycentric_2d(q_w)
        w_inv = np.linalg.inv(el.mono(lam_w @ el.X, q_w))
        wc = w_inv @ conv                                   # monomial coefficients of w
        wq_v = el.mono(xq, q_w) @ wc                        # w at volume points
        # -(u, (w·∇)v): rows v_i, cols u_j
        wgrad = np.einsum("qicd,qd->qic", GU, wq_v)         # ((w·∇)φ_i)_c
        Cv = np.zeros((n, n))
        Cv[ou:ou + nrt, ou:ou + nrt] -= np.einsum("q,qic,qjc->ij", wq, wgrad, U)
        nF = upwind_facet_points(k, q_w)
        for f in range(3):
            fd = el.facets[f]
            s, xf, wf = el.facet_points(f, nF)
            nK = fd["nK"]
            wn = (el.mono(xf, q_w) @ wc) @ nK
            wp, wm = np.maximum(wn, 0.0), np.minimum(wn, 0.0)
            Uf = el.rt_values(xf)
            tngU = Uf - np.einsum("qi,c->qic", Uf @ nK, nK)
            lm = el.facet_legendre(f, s)
            Hf = np.einsum("qm,c->qmc", lm, fd["t"])       # û basis on this facet
            hs = slice(oh + f * (k + 1), oh + (f + 1) * (k + 1))
            Cv[ou:ou + nrt, ou:ou + nrt] += np.einsum("q,qic,qjc->ij", wf * wp, tngU, tngU)
            Cv[ou:ou + nrt, hs] += np.einsum("q,qic,qmc->im", wf * wm, tngU, Hf)
            Cv[hs, ou:ou + nrt] -= np.einsum("q,qmc,qjc->mj", wf * wp, Hf, tngU)
            Cv[hs, hs] -= np.einsum("q,qmc,qnc->mn", wf * wm, Hf, Hf)
        M += Cv.T if conv_transpose else Cv
        if newton_uhat is not None:
            uh = np.asarray(newton_uhat, dtype=float)
            Cp = np.zeros((n, n))
            # -(u_old, (φ_j·∇)φ_i): rows v_i, cols δu_j
            Cp[ou:ou + nrt, ou:ou + nrt] -= np.einsum("q,qc,qjd,qicd->ij", wq, wq_v, U, GU)
            extra = np.zeros(n)
            extra[ou:ou + nrt] -= np.einsum("q,qc,qd,qicd->i", wq, wq_v, wq_v, GU)
            for f in range(3):
                fd = el.facets[f]
                s_, xf, wf = el.facet_points(f, nF)
                nK = fd["nK"]
                wf_v = el.mono(xf, q_w) @ wc                           # u_old at the facet points
                an = wf_v @ nK
                lm = el.facet_legendre(f, s_)
                Hf = np.einsum("qm,c->qmc", lm, fd["t"])
                tng_old = wf_v - np.outer(an, nK)
                tng_hat = np.einsum("qm,m,c->qc", lm, uh[f], fd["t"])
                # ties: where |w·n| is at rounding level (Dirichlet facets, symmetric nodes)
                # the trace of û is taken, so the switch does not follow rounding noise
                up = (an > NEWTON_TIE * np.abs(conv).max()) & (not newton_boundary[f])
                wup = np.where(up[:, None], tng_old, tng_hat)
                Uf = el.rt_values(xf)
                nU = Uf @ nK                                             # (q, nrt) φ_j·n_K
                tngU = Uf - np.einsum("qi,c->qic", nU, nK)
                hs = slice(oh + f * (k + 1), oh + (f + 1) * (k + 1))
                Cp[ou:ou + nrt, ou:ou + nrt] += np.einsum("q,qj,qc,qic->ij", wf, nU, wup, tngU)
                Cp[hs, ou:ou + nrt] -= np.einsum("q,qj,qc,qmc->mj", wf, nU, wup, Hf)
                extra[ou:ou + nrt] += np.einsum("q,q,qc,qic->i", wf, an, wup, tngU)
                extra[hs] -= np.einsum("q,q,qc,qmc->m", wf, an, wup, Hf)
            M += Cp
    # forcing: f_h ∈ [P^{k+1}]² from its values at the degree-(k+1) lattice
    lam = lattice_barycentric_2d(k + 1)
    Xl = lam @ el.X
    lat_inv = np.linalg.inv(el.mono(Xl, k + 1))
    Lq = el.mono(xq, k + 1) @ lat_inv                     # (q, n_lat) lattice Lagrange values
    Rf = np.einsum("q,qn,qic->inc", wq, Lq, U).reshape(nrt, -1)
    rhs_map = np.zeros((n, Rf.shape[1]))
    rhs_map[ou:ou + nrt] = Rf
    g = []
    for f in range(3):
        g += [ou + f * (k + 1) + m for m in range(k + 1)]
        g += [oh + f * (k + 1) + m for m in range(k + 1)]
    loc = list(range(oL, oL + nL)) + list(range(ou + 3 * (k + 1), ou + nrt)) + \
        list(range(op + 1, op + npp))
    info = dict(oL=oL, ou=ou, oh=oh, op=op, npk=npk, nrt=nrt)
    if conv is not None and newton_uhat is not None:
        info["rhs_extra"] = extra
    return M, rhs_map, np.asarray(g), np.asarray(loc), op, lat_inv, info


def condense_cell(el: Element, nu: float, beta: float, conv=None,
                  conv_transpose: bool = False, newton_uhat=None,
                  newton_boundary=(False, False, False)) -> CondensedCell:
    """Static condensation of one cell by a dense Schur complement."""
    return schur_condense(el, *local_system(el, nu, beta, conv, conv_transpose, newton_uhat,
                                            newton_boundary))


def schur_condense(el, M, rhs_map, g, loc, p0, lat_inv, info) -> CondensedCell:
    """Eliminate the local unknowns `loc` of the full local system M (the dense Schur
    complement onto the facet unknowns `g`; the cell-mean pressure p0 stays global)."""
    Mll = M[np.ix_(loc, loc)]
    Mlg = M[np.ix_(loc, g)]
    Mgl = M[np.ix_(g, loc)]
    extra = info.get("rhs_extra")
    cols = [Mlg, M[loc, p0][:, None], rhs_map[loc]]
    if extra is not None:
        cols.append(extra[loc][:, None])
    X = np.linalg.solve(Mll, np.hstack(cols))
    ng = len(g)
    nf = rhs_map.shape[1]
    Xg, Xp, Xf = X[:, :ng], X[:, ng], X[:, ng + 1:ng + 1 + nf]
    A = M[np.ix_(g, g)] - Mgl @ Xg
    d = M[p0, g] - M[p0, loc] @ Xg
    Fmap = rhs_map[g] - Mgl @ Xf
    Fextra = Rextra = None
    if extra is not None:
        Rextra = X[:, ng + 1 + nf]
        Fextra = extra[g] - Mgl @ Rextra
    return CondensedCell(A=A, d=d, Fmap=Fmap, area=el.area, Rf=Xf, Rg=Xg, Rp=Xp,
                         el=el, lat_inv=lat_inv, Fextra=Fextra, Rextra=Rextra)


class HDG:
    """Condensed H(div)-HDG operator of order k on one mesh level."""

    def __init__(self, topo: Topology, k: int, nu: float = 1.0, beta: float = 0.0,
                 gamma: float = 0.0, nu_elem: Optional[np.ndarray] = None,
                 cache: bool = True, conv: Optional[np.ndarray] = None,
                 conv_transpose: bool = False, newton_uhat: Optional[np.ndarray] = None,
                 dirichlet: Optional[np.ndarray] = None):
        """dirichlet: the skeleton values of inhomogeneous Dirichlet data, (n_boundary_facets,
        2(k+1)) in facet order (boundary facets only), the unknowns' layout (normal moments,
        then tangential coefficients); None = homogeneous data."""
        self.topo, self.k = topo, k
        self.dpf = 2 * (k + 1)
        self.ng = 3 * self.dpf
        self.nu = float(nu)
        self.beta = float(beta)
        self.gamma = float(gamma)
        nc = topo.n_cells
        self.nu_elem = np.full(nc, self.nu) if nu_elem is None else np.asarray(nu_elem, float)
        self.n_dof = topo.n_interior * self.dpf
        self.conv = None if conv is None else np.asarray(conv, dtype=float)
        self.conv_transpose = bool(conv_transpose)
        self.newton_uhat = None if newton_uhat is None else np.asarray(newton_uhat, dtype=float)
        if self.newton_uhat is not None:
            cache = False
        self.cells = []
        memo = {}
        for c in range(nc):
            gv = topo.cells[c]
            X = topo.coords[gv]
            cv = None if self.conv is None else self.conv[c]
            key = _signature(X, gv, k, self.nu_elem[c], beta, cv, conv_transpose) if cache else None
            if key is not None and key in memo:
                cc = memo[key]
            else:
                el = Element(X - X[0], gv, k)
                nh = None if self.newton_uhat is None else self.newton_uhat[c]
                bnd = tuple(bool(topo.interior_index[topo.cell_facets[c, f]] < 0) for f in range(3))
                cc = condense_cell(el, self.nu_elem[c], beta, cv, conv_transpose, nh, bnd)
                if key is not None:
                    memo[key] = cc
            self.cells.append(cc)
        self.area = np.array([cc.area for cc in self.cells])
        self.eps_inv = self.gamma * self.nu_elem
        # local → global unknown map (−1 for boundary facets)
        self.l2g = -np.ones((nc, self.ng), dtype=np.int64)
        for c in range(nc):
            for f in range(3):
                i = topo.interior_index[topo.cell_facets[c, f]]
                if i >= 0:
                    self.l2g[c, f * self.dpf:(f + 1) * self.dpf] = i * self.dpf + np.arange(self.dpf)
        # boundary data: local unknowns of boundary facets -> entries of the data vector
        bnd_facets = np.flatnonzero(topo.interior_index < 0)
        self.n_boundary = len(bnd_facets)
        self.xD = None
        self.b2g = -np.ones((nc, self.ng), dtype=np.int64)
        if dirichlet is not None:
            data = np.asarray(dirichlet, dtype=float)
            assert data.shape == (self.n_boundary, self.dpf), "dirichlet: (n_boundary_facets, dpf)"
            self.xD = data.reshape(-1)
            bidx = -np.ones(len(topo.interior_index), dtype=np.int64)
            bidx[bnd_facets] = np.arange(self.n_boundary)
            for c in range(nc):
                for f in range(3):
                    b = bidx[topo.cell_facets[c, f]]
                    if b >= 0:
                        self.b2g[c, f * self.dpf:(f + 1) * self.dpf] = b * self.dpf + np.arange(self.dpf)

    # ------------------------------------------------------------ element data
    def element_matrix(self, c: int, with_al: bool = True) -> np.ndarray:
        cc = self.cells[c]
        A = cc.A.copy()
        if with_al:
            A += (self.eps_inv[c] / cc.area) * np.outer(cc.d, cc.d)
        return A

    def element_load(self, c: int, fvals_c: np.ndarray) -> np.ndarray:
        cc = self.cells[c]
        F = cc.Fmap @ np.asarray(fvals_c).reshape(-1)
        return F if cc.Fextra is None else F + cc.Fextra

    # ------------------------------------------------------------ global
    def matrix(self, with_al: bool = True) -> sp.csr_matrix:
        rows, cols, vals = [], [], []
        for c in range(self.topo.n_cells):
            idx = self.l2g[c]
            m = idx >= 0
            A = self.element_matrix(c, with_al)[np.ix_(m, m)]
            I = idx[m]
            rows.append(np.repeat(I, len(I)))
            cols.append(np.tile(I, len(I)))
            vals.append(A.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_dof, self.n_dof))

    def flux_matrix(self) -> sp.csr_matrix:
        """D (n_cells × n_dof): (D u)_K = ∫_{∂K} u·n_K = |K| (div u)_K."""
        rows, cols, vals = [], [], []
        for c in range(self.topo.n_cells):
            idx = self.l2g[c]
            m = idx >= 0
            rows.append(np.full(int(m.sum()), c))
            cols.append(idx[m])
            vals.append(self.cells[c].d[m])
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.topo.n_cells, self.n_dof))

    def local_dirichlet(self, c: int) -> np.ndarray:
        """Cell c's local unknowns carrying Dirichlet data (zero on interior facets)."""
        out = np.zeros(self.ng)
        if self.xD is not None:
            b = self.b2g[c]
            out[b >= 0] = self.xD[b[b >= 0]]
        return out

    def load(self, fvals: np.ndarray) -> np.ndarray:
        """Condensed load F (n_dof,) from lattice forcing (n_cells, n_lat, 2), minus the
        coupling of the interior unknowns to the Dirichlet data through A^ε."""
        F = np.zeros(self.n_dof)
        for c in range(self.topo.n_cells):
            idx = self.l2g[c]
            m = idx >= 0
            Fc = self.element_load(c, fvals[c])
            if self.xD is not None:
                Fc = Fc - self.element_matrix(c) @ self.local_dirichlet(c)
            F[idx[m]] += Fc[m]
        return F

    def boundary_flux(self) -> np.ndarray:
        """Per cell, the flux of the Dirichlet data through its boundary facets (the part of
        |K| div u_h that the interior unknowns do not carry)."""
        if self.xD is None:
            return np.zeros(self.topo.n_cells)
        return np.array([self.cells[c].d @ self.local_dirichlet(c) for c in range(self.topo.n_cells)])

    def gather(self, x: np.ndarray, c: int) -> np.ndarray:
        idx = self.l2g[c]
        out = self.local_dirichlet(c)
        out[idx >= 0] = x[idx[idx >= 0]]
        return out

    def facet_tangential(self, x: np.ndarray) -> np.ndarray:
        """(n_cells, 3, k+1): each cell's facet tangential coefficients of the skeleton vector x."""
        out = np.zeros((self.topo.n_cells, 3, self.k + 1))
        for c in range(self.topo.n_cells):
            xg = self.gather(x, c)
            for f in range(3):
                out[c, f] = xg[f * self.dpf + self.k + 1:(f + 1) * self.dpf]
        return out

    # ------------------------------------------------------------ exact solve
    def solve_direct(self, F: np.ndarray):
        """Exact discrete solution of A u − Dᵀp = F, D u + b = 0, Σ|K|p_K = 0 (b: the
        cells' boundary fluxes of the Dirichlet data, zero for homogeneous data).

        The condensed saddle point of eq. stOptForm (the B-rows are the cell
        fluxes; the mean-zero pressure is imposed by one Lagrange multiplier).
        Returns (u (n_dof,), p (n_cells,)).
        """
        A = self.matrix(with_al=False)
        D = self.flux_matrix()
        nc = self.topo.n_cells
        w = sp.csr_matrix(self.area[:, None])
        K = sp.bmat([[A, -D.T, None], [D, None, w], [None, w.T, None]], format="csc")
        bf = self.boundary_flux()
        # F carries -A^ε_IB u_D; without the AL term the load is F + eps^-1 d_I (d_B u_D) / |K|
        Fn = F + D.T @ (self.eps_inv * bf / self.area)
        rhs = np.concatenate([Fn, -bf, [0.0]])
        sol = spla.splu(K).solve(rhs)
        return sol[:self.n_dof], sol[self.n_dof:self.n_dof + nc]

    def solve_al_exact(self, F: np.ndarray, tol: float = 1e-13, max_steps: int = 60):
        """The same discrete solution by the augmented-Lagrangian Uzawa iteration of Section 3.3
        with exact inner solves (one sparse LU of A^ε): p ← p − ε⁻¹|K|⁻¹ D u, which contracts by
        about 1/(1+γ) per step (Lemma 3.1); stops when |D u|/|F| < tol.  Homogeneous data only.
        For meshes where the LU of the saddle-point matrix fills in too much (3D)."""
        assert self.xD is None
        lu = spla.splu(self.matrix(with_al=True).tocsc())
        D = self.flux_matrix()
        p = np.zeros(self.topo.n_cells)
        nF = np.linalg.norm(F)
        for _ in range(max_steps):
            u = lu.solve(F + D.T @ p)
            du = D @ u
            if np.linalg.norm(du) <= tol * nF:
                break
            p -= self.eps_inv * du / self.area
        return u, p - (self.area @ p) / self.area.sum()

    # ------------------------------------------------------------ recovery
    def recover_cell(self, c: int, u: np.ndarray, pK: float, fvals_c: np.ndarray):
        """Local fields on cell c: (L coeffs (4, npk), RT coeffs (n_rt,), p coeffs (npk,))."""
        cc = self.cells[c]
        k = self.k
        npk = len(exponents(k))
        xg = self.gather(u, c)
        y = cc.Rf @ np.asarray(fvals_c).reshape(-1) - cc.Rg @ xg - cc.Rp * pK
        if cc.Rextra is not None:
            y = y + cc.Rextra
        nL = 4 * npk
        Lc = y[:nL].reshape(4, npk)
        nrt = cc.el.n_rt
        rt = np.zeros(nrt)
        for f in range(3):
            rt[f * (k + 1):(f + 1) * (k + 1)] = xg[f * self.dpf:f * self.dpf + k + 1]
        n_int = nrt - 3 * (k + 1)
        rt[3 * (k + 1):] = y[nL:nL + n_int]
        pc = np.concatenate([[pK], y[nL + n_int:]])
        return Lc, rt, pc

    def fields_at(self, c, coeffs, xq):
        """Evaluate (L (q,2,2), u (q,2), div u (q,), p (q,)) at points xq (translated)."""
        Lc, rt, pc = coeffs
        el = self.cells[c].el
        Pk = el.mono(xq, self.k)
        L = np.einsum("qr,cr->qc", Pk, Lc).reshape(-1, 2, 2)
        U = el.rt_values(xq)
        u = np.einsum("qic,i->qc", U, rt)
        divu = el.rt_div(xq) @ rt
        # pressure basis: 1 and mean-free monomials (same as in local_system)
        xq2, wq2 = triangle_points(el.X, self.k + 3)
        mean = (wq2 @ el.mono(xq2, self.k)) / el.area
        pv = Pk - mean[None, :]
        pv[:, 0] = 1.0
        p = pv @ pc
        return L, u, divu, p

    def ustar_cell(self, c: int, coeffs, nq: Optional[int] = None) -> np.ndarray:
        """Post-processed u* ∈ [P^{k+1}]² on cell c (eq. stPost, read with L = −ν∇u):
        (∇u*, ∇v)_K = (−ν⁻¹L_h, ∇v)_K for v ∈ P^{k+1} except the constant, whose
        equation is replaced by (u*, 1)_K = (u_h, 1)_K.  Returns the coefficients over
        the cell's monomials of degree <= k+1, shape (n_mono, 2)."""
        k = self.k
        el = self.cells[c].el
        xq, wq = triangle_points(el.X, nq or (k + 5))
        L, uh, _, _ = self.fields_at(c, coeffs, xq)
        Gm = el.mono_grad(xq, k + 1)
        Mo = el.mono(xq, k + 1)
        S = np.einsum("q,qid,qjd->ij", wq, Gm, Gm)
        S[0, :] = wq @ Mo
        us = np.zeros((Mo.shape[1], 2))
        for a in range(2):
            r = np.einsum("q,qid,qd->i", wq, Gm, -L[:, a, :] / self.nu_elem[c])
            r[0] = wq @ uh[:, a]
            us[:, a] = np.linalg.solve(S, r)
        return us

    def postprocess(self, u, p, fvals) -> np.ndarray:
        """u* at every cell's degree-(k+1) lattice (the forcing layout): (n_cells, n_lat, 2)."""
        lam = lattice_barycentric_2d(self.k + 1)
        out = np.zeros((self.topo.n_cells, lam.shape[0], 2))
        for c in range(self.topo.n_cells):
            coeffs = self.recover_cell(c, u, p[c], fvals[c])
            el = self.cells[c].el
            out[c] = el.mono(lam @ el.X, self.k + 1) @ self.ustar_cell(c, coeffs)
        return out

    def errors(self, u, p, fvals, sol, nq: Optional[int] = None):
        """L2 errors of u_h, L_h (L = −ν∇u), p_h (both mean-free), ‖div u_h‖, and u*.

        The post-processed u* ∈ [P^{k+1}]² solves, per cell,
        (∇u*, ∇v)_K = (−ν⁻¹L_h, ∇v)_K and (u*, 1)_K = (u_h, 1)_K (eq. stPost,
        read with L = −ν∇u so that ∇u* approximates ∇u).
        """
        k = self.k
        nq = nq or (k + 5)
        eu = eL = ediv = eus = 0.0
        pint = pex_int = 0.0
        ph_vals, pe_vals, wts = [], [], []
        for c in range(self.topo.n_cells):
            X0 = self.topo.coords[self.topo.cells[c][0]]
            el = self.cells[c].el
            xq, wq = triangle_points(el.X, nq)
            coeffs = self.recover_cell(c, u, p[c], fvals[c])
            L, uh, divu, ph = self.fields_at(c, coeffs, xq)
            xa = xq + X0
            ue = sol.u(xa)
            Le = -self.nu_elem[c] * sol.grad_u(xa)
            eu += wq @ np.sum((ue - uh) ** 2, axis=1)
            eL += wq @ np.sum((Le - L) ** 2, axis=(1, 2))
            ediv += wq @ divu ** 2
            ph_vals.append(ph)
            pe_vals.append(sol.p(xa))
            wts.append(wq)
            # post-processing u* in [P^{k+1}]^2
            ustar = el.mono(xq, k + 1) @ self.ustar_cell(c, coeffs, nq)
            eus += wq @ np.sum((ue - ustar) ** 2, axis=1)
        ph = np.concatenate(ph_vals)
        pe = np.concatenate(pe_vals)
        w = np.concatenate(wts)
        ph = ph - (w @ ph) / w.sum()
        pe = pe - (w @ pe) / w.sum()
        ep = np.sqrt(w @ (ph - pe) ** 2)
        return dict(u=np.sqrt(eu), L=np.sqrt(eL), p=ep, div=np.sqrt(ediv), ustar=np.sqrt(eus))
