"""H(div)-HDG on tetrahedra: local systems, static condensation, exact discrete solution.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The scheme of Section 3.2 (eq. stWeak) with d = 3: find (L_h, u_h, û_h, p_h) in
[W^k]^{3×3} × RT_k × V̂^k × W^k with, on every cell,
  (ν⁻¹L, G) + (∇u, G) − ⟨tng(u − û), G n⟩                      = 0,
  −(L, ∇v) + ⟨L n, tng(v − v̂)⟩ + β(u, v) − (p, div v)           = (f, v),
  (div u, q)                                                        = 0,
written by quadrature in physical coordinates and condensed by a dense Schur
complement onto the face unknowns (the same route as the 2D oracle).  What
remains per cell is A_K on the 4·dpf face unknowns, dpf = 3(k+1)(k+2)/2: per
face the nf = (k+1)(k+2)/2 normal moments, then the t1 and the t2 coefficients of
the tangential unknown (frames and bases in oracle/spaces3d.py); the flux row d_K
and the augmented-Lagrangian term ε⁻¹|K|⁻¹ d_K d_Kᵀ, ε⁻¹ = γν, as in 2D.
Generalized Stokes only (no convection) in 3D.
"""

from __future__ import annotations

from typing import Optional

import numpy as np

from workloads.manufactured import lattice_barycentric_3d

from .hdg import HDG, _signature, schur_condense
from .quadrature import face_points, tetrahedron_points
from .spaces3d import Element3, exponents3, face_data, face_mono, n_face
from .topology3d import Topology3D


def local_system_3d(el: Element3, nu: float, beta: float):
    """Full local matrix over (L, u, û, p) on a tetrahedron, forcing map and index sets
    (the layout of oracle.hdg.local_system's return value)."""
    k = el.k
    npk = len(exponents3(k))
    nf = el.nf
    nL, nrt, nh, npp = 9 * npk, el.n_rt, 8 * nf, npk
    oL, ou, oh, op = 0, nL, nL + nrt, nL + nrt + nh
    n = op + npp
    M = np.zeros((n, n))
    xq, wq = tetrahedron_points(el.X, k + 3)
    Pk = el.mono(xq, k)
    mean = (wq @ Pk) / el.vol
    pv = Pk - mean[None, :]
    pv[:, 0] = 1.0                      # exponents3(k)[0] == (0, 0, 0): global P0 part
    U = el.rt_values(xq)
    GU = el.rt_grads(xq)
    DU = GU[:, :, 0, 0] + GU[:, :, 1, 1] + GU[:, :, 2, 2]
    Mp = (Pk * wq[:, None]).T @ Pk
    for ce in range(9):
        M[oL + ce * npk:oL + (ce + 1) * npk, oL + ce * npk:oL + (ce + 1) * npk] = Mp / nu
    for c in range(3):
        for e in range(3):
            ce = 3 * c + e
            M[oL + ce * npk:oL + (ce + 1) * npk, ou:ou + nrt] += (Pk * wq[:, None]).T @ GU[:, :, c, e]
    for f in range(4):
        fd = el.facets[f]
        xf, lm, wf = el.face_quad(f, k + 3)
        Uf = el.rt_values(xf)
        nK = fd["nK"]
        tngU = Uf - np.einsum("qi,c->qic", Uf @ nK, nK)
        Pf = el.mono(xf, k)
        for c in range(3):
            for e in range(3):
                ce = 3 * c + e
                rows = slice(oL + ce * npk, oL + (ce + 1) * npk)
                M[rows, ou:ou + nrt] -= (Pf * (wf * nK[e])[:, None]).T @ tngU[:, :, c]
                for a, t in enumerate((fd["t1"], fd["t2"])):
                    cols = slice(oh + f * 2 * nf + a * nf, oh + f * 2 * nf + (a + 1) * nf)
                    M[rows, cols] += (Pf * (wf * nK[e] * t[c])[:, None]).T @ lm
    M[ou:ou + nrt, oL:oL + nL] = -M[oL:oL + nL, ou:ou + nrt].T
    M[oh:oh + nh, oL:oL + nL] = -M[oL:oL + nL, oh:oh + nh].T
    M[ou:ou + nrt, ou:ou + nrt] += beta * np.einsum("q,qic,qjc->ij", wq, U, U)
    Bd = np.einsum("q,qi,qj->ij", wq, DU, pv)
    M[ou:ou + nrt, op:op + npp] = -Bd
    M[op:op + npp, ou:ou + nrt] = Bd.T
    # forcing: f_h ∈ [P^{k+1}]³ from its values at the degree-(k+1) lattice
    lam = lattice_barycentric_3d(k + 1)
    lat_inv = np.linalg.inv(el.mono(lam @ el.X, k + 1))
    Lq = el.mono(xq, k + 1) @ lat_inv
    Rf = np.einsum("q,qn,qic->inc", wq, Lq, U).reshape(nrt, -1)
    rhs_map = np.zeros((n, Rf.shape[1]))
    rhs_map[ou:ou + nrt] = Rf
    g = []
    for f in range(4):
        g += [ou + f * nf + m for m in range(nf)]
        g += [oh + f * 2 * nf + j for j in range(2 * nf)]
    loc = list(range(oL, oL + nL)) + list(range(ou + 4 * nf, ou + nrt)) + list(range(op + 1, op + npp))
    info = dict(oL=oL, ou=ou, oh=oh, op=op, npk=npk, nrt=nrt)
    return M, rhs_map, np.asarray(g), np.asarray(loc), op, lat_inv, info


def condense_cell_3d(el: Element3, nu: float, beta: float):
    return schur_condense(el, *local_system_3d(el, nu, beta))


class HDG3D(HDG):
    """Condensed H(div)-HDG operator of order k on one tetrahedral mesh level (generalized
    Stokes).  The global methods (assembly, flux rows, loads, the exact saddle-point solve)
    are the 2D class's, which only see cells, local-to-global maps and the cell measures."""

    def __init__(self, topo: Topology3D, k: int, nu: float = 1.0, beta: float = 0.0,
                 gamma: float = 0.0, nu_elem: Optional[np.ndarray] = None, cache: bool = True,
                 dirichlet: Optional[np.ndarray] = None):
        self.topo, self.k = topo, k
        self.nfb = n_face(k)
        self.dpf = 3 * self.nfb
        self.ng = 4 * self.dpf
        self.nu, self.beta, self.gamma = float(nu), float(beta), float(gamma)
        nc = topo.n_cells
        self.nu_elem = np.full(nc, self.nu) if nu_elem is None else np.asarray(nu_elem, float)
        self.n_dof = topo.n_interior * self.dpf
        self.conv = None
        self.conv_transpose = False
        self.newton_uhat = None
        self.cells = []
        memo = {}
        for c in range(nc):
            gv = topo.cells[c]
            X = topo.coords[gv]
            key = _signature(X, gv, k, self.nu_elem[c], beta) if cache else None
            if key is not None and key in memo:
                cc = memo[key]
            else:
                cc = condense_cell_3d(Element3(X - X[0], gv, k), self.nu_elem[c], beta)
                if key is not None:
                    memo[key] = cc
            self.cells.append(cc)
        self.area = np.array([cc.area for cc in self.cells])
        self.eps_inv = self.gamma * self.nu_elem
        self.l2g = -np.ones((nc, self.ng), dtype=np.int64)
        for c in range(nc):
            for f in range(4):
                i = topo.interior_index[topo.cell_facets[c, f]]
                if i >= 0:
                    self.l2g[c, f * self.dpf:(f + 1) * self.dpf] = i * self.dpf + np.arange(self.dpf)
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
                for f in range(4):
                    b = bidx[topo.cell_facets[c, f]]
                    if b >= 0:
                        self.b2g[c, f * self.dpf:(f + 1) * self.dpf] = b * self.dpf + np.arange(self.dpf)

    # ------------------------------------------------------------ recovery
    def recover_cell(self, c: int, u: np.ndarray, pK: float, fvals_c: np.ndarray):
        """Local fields on cell c: (L coeffs (9, npk), RT coeffs (n_rt,), p coeffs (npk,))."""
        cc = self.cells[c]
        npk = len(exponents3(self.k))
        nf = self.nfb
        xg = self.gather(u, c)
        y = cc.Rf @ np.asarray(fvals_c).reshape(-1) - cc.Rg @ xg - cc.Rp * pK
        nL = 9 * npk
        Lc = y[:nL].reshape(9, npk)
        nrt = cc.el.n_rt
        rt = np.zeros(nrt)
        for f in range(4):
            rt[f * nf:(f + 1) * nf] = xg[f * self.dpf:f * self.dpf + nf]
        n_int = nrt - 4 * nf
        rt[4 * nf:] = y[nL:nL + n_int]
        pc = np.concatenate([[pK], y[nL + n_int:]])
        return Lc, rt, pc

    def fields_at(self, c, coeffs, xq):
        """(L (q,3,3), u (q,3), div u (q,), p (q,)) at points xq (translated coordinates)."""
        Lc, rt, pc = coeffs
        el = self.cells[c].el
        Pk = el.mono(xq, self.k)
        L = np.einsum("qr,cr->qc", Pk, Lc).reshape(-1, 3, 3)
        u = np.einsum("qic,i->qc", el.rt_values(xq), rt)
        divu = el.rt_div(xq) @ rt
        xq2, wq2 = tetrahedron_points(el.X, self.k + 3)
        mean = (wq2 @ el.mono(xq2, self.k)) / el.vol
        pv = Pk - mean[None, :]
        pv[:, 0] = 1.0
        return L, u, divu, pv @ pc

    def ustar_cell(self, c: int, coeffs, nq: Optional[int] = None) -> np.ndarray:
        """Post-processed u* ∈ [P^{k+1}]³ on cell c (eq. stPost, read with L = −ν∇u):
        (∇u*, ∇v)_K = (−ν⁻¹L_h, ∇v)_K for v ∈ P^{k+1} except the constant, whose equation is
        replaced by (u*, 1)_K = (u_h, 1)_K.  Coefficients over the cell's monomials of degree
        <= k+1, shape (n_mono, 3)."""
        k = self.k
        el = self.cells[c].el
        xq, wq = tetrahedron_points(el.X, nq or (k + 4))
        L, uh, _, _ = self.fields_at(c, coeffs, xq)
        Gm = el.mono_grad(xq, k + 1)
        Mo = el.mono(xq, k + 1)
        S = np.einsum("q,qid,qjd->ij", wq, Gm, Gm)
        S[0, :] = wq @ Mo
        us = np.zeros((Mo.shape[1], 3))
        for a in range(3):
            r = np.einsum("q,qid,qd->i", wq, Gm, -L[:, a, :] / self.nu_elem[c])
            r[0] = wq @ uh[:, a]
            us[:, a] = np.linalg.solve(S, r)
        return us

    def postprocess(self, u, p, fvals) -> np.ndarray:
        """u* at every cell's degree-(k+1) lattice (the forcing layout): (n_cells, n_lat, 3)."""
        lam = lattice_barycentric_3d(self.k + 1)
        out = np.zeros((self.topo.n_cells, lam.shape[0], 3))
        for c in range(self.topo.n_cells):
            el = self.cells[c].el
            out[c] = el.mono(lam @ el.X, self.k + 1) @ self.ustar_cell(c, self.recover_cell(c, u, p[c], fvals[c]))
        return out

    def errors(self, u, p, fvals, sol, nq: Optional[int] = None):
        """L2 errors of u_h, L_h (L = −ν∇u), p_h (both mean-free) and ‖div u_h‖."""
        nq = nq or (self.k + 4)
        eu = eL = ediv = 0.0
        ph_vals, pe_vals, wts = [], [], []
        for c in range(self.topo.n_cells):
            X0 = self.topo.coords[self.topo.cells[c][0]]
            el = self.cells[c].el
            xq, wq = tetrahedron_points(el.X, nq)
            L, uh, divu, ph = self.fields_at(c, self.recover_cell(c, u, p[c], fvals[c]), xq)
            xa = xq + X0
            eu += wq @ np.sum((sol.u(xa) - uh) ** 2, axis=1)
            eL += wq @ np.sum((-self.nu_elem[c] * sol.grad_u(xa) - L) ** 2, axis=(1, 2))
            ediv += wq @ divu ** 2
            ph_vals.append(ph)
            pe_vals.append(sol.p(xa))
            wts.append(wq)
        ph, pe, w = np.concatenate(ph_vals), np.concatenate(pe_vals), np.concatenate(wts)
        ph = ph - (w @ ph) / w.sum()
        pe = pe - (w @ pe) / w.sum()
        return dict(u=np.sqrt(eu), L=np.sqrt(eL), p=np.sqrt(w @ (ph - pe) ** 2), div=np.sqrt(ediv))


def dirichlet_data_3d(topo: Topology3D, k: int, g, nq: Optional[int] = None) -> np.ndarray:
    """Skeleton values (n_boundary, dpf) of boundary data g on the boundary faces in face
    order, in the unknowns' layout: ∫_F (g·n_F) ℓ_m, then ∫_F (g·t1) ℓ_m and ∫_F (g·t2) ℓ_m."""
    nq = nq or (k + 5)
    out = []
    for F in np.flatnonzero(topo.interior_index < 0):
        fd = face_data(topo.coords[topo.facets[F]], k)
        x, ref, w = face_points(fd["Xf"], nq)
        lm = face_mono(ref, k) @ fd["orth"]
        gv = g(x)
        out.append(np.concatenate([(w * (gv @ v)) @ lm for v in (fd["nF"], fd["t1"], fd["t2"])]))
    return np.asarray(out)
