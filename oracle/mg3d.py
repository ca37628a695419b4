"""Edge-patch smoothers, intergrid transfer and hp-multigrid on tetrahedra (oracle).

TEST INFRASTRUCTURE ONLY.  The 3D counterparts of oracle/mg.py, on assembled global
sparse matrices with plain sequential loops:

* Edge patches (Section 3.4.2: in three dimensions the block smoother may use edge
  patches to save memory): the patch of edge e holds every unknown on the interior
  faces containing e; patches are visited by colour, then by edge id
  (oracle/topology3d.py).  Block GS and damped block Jacobi are oracle/mg.py's.
* Averaging transfer I_{l−1}^l (eq. avgOpt) with 3 unknowns per face: Π^CR of the
  coarse function (ψ_i = 1 − 3λ_i, barycentre values (c_n n + c_1 t1 + c_2 t2)/sqrt|F|)
  at each fine face barycentre; inside a coarse cell that cell's value, on a coarse
  face the mean of the two sides.
* Harmonic-extension correction (eqs. div-transfer, harmonic-ex) and Algorithms 1
  and 2: oracle/mg.py's, with Π_0^k the injection of the m = 0 normal, t1 and t2
  coefficients of each face.
"""

from __future__ import annotations

from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .cr3d import bary_3d
from .hdg3d import HDG3D
from .mg import MGh, MGhp, harmonic_prolongation, make_smoother
from .topology3d import Topology3D, edge_patches


def averaging_prolongation_3d(coarse: Topology3D, fine: Topology3D, parent: np.ndarray) -> sp.csr_matrix:
    """I_{l−1}^l of eq. avgOpt on lowest-order unknowns (3 per interior face)."""
    rows, cols, vals = [], [], []

    def cr_weights(Kc, x):
        lam = bary_3d(coarse.coords[coarse.cells[Kc]], x)[0]
        out = []
        for i in range(4):
            ii = coarse.interior_index[coarse.cell_facets[Kc, i]]
            if ii < 0:
                continue
            _, _, _, area, t1, t2, nF = coarse.facet_geometry(coarse.cell_facets[Kc, i])
            psi = 1.0 - 3.0 * lam[i]
            for a, v in enumerate((nF, t1, t2)):
                out.append((3 * ii + a, psi * v / np.sqrt(area)))
        return out

    for i, F in enumerate(fine.interior_facets):
        c0, c1 = fine.facet_cells[F]
        xa, xb, xc, area, t1, t2, nF = fine.facet_geometry(F)
        mid = (xa + xb + xc) / 3.0
        p0, p1 = parent[c0], parent[c1]
        sides = [p0] if p0 == p1 else [p0, p1]
        w = 1.0 / len(sides)
        for Kc in sides:
            for col, vec in cr_weights(Kc, mid):
                for a, v in enumerate((nF, t1, t2)):
                    rows.append(3 * i + a)
                    cols.append(col)
                    vals.append(w * np.sqrt(area) * (vec @ v))
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * fine.n_interior, 3 * coarse.n_interior))


def interior_fine_dofs_3d(fine: Topology3D, parent: np.ndarray) -> np.ndarray:
    """Lowest-order unknowns on fine faces inside coarse cells (the set T)."""
    out = []
    for i, F in enumerate(fine.interior_facets):
        c0, c1 = fine.facet_cells[F]
        if parent[c0] == parent[c1]:
            out += [3 * i, 3 * i + 1, 3 * i + 2]
    return np.asarray(out, dtype=np.int64)


class Level3D:
    def __init__(self, hdg: HDG3D, smoother: str = "gs", damping: float = 0.5):
        self.hdg = hdg
        self.A = hdg.matrix(with_al=True).tocsr()
        self.gs = make_smoother(self.A, edge_patches(hdg.topo, hdg.dpf), smoother, damping)
        self.P: Optional[sp.csr_matrix] = None


class MGh3D(MGh):
    """Algorithm 1 on tetrahedral lowest-order levels (index 0 = coarsest)."""

    def __init__(self, levels: List[Level3D], parents: List[np.ndarray], growth: int = 2):
        self.levels = levels
        self.growth = growth
        for l in range(1, len(levels)):
            Ia = averaging_prolongation_3d(levels[l - 1].hdg.topo, levels[l].hdg.topo, parents[l])
            T = interior_fine_dofs_3d(levels[l].hdg.topo, parents[l])
            levels[l].P = harmonic_prolongation(levels[l].A, Ia, T)
        self.symmetric = True
        self.coarse = sla.cho_factor(levels[0].A.toarray())


def inclusion_matrix_3d(n_int: int, k: int) -> sp.csr_matrix:
    """Π_0^k: lowest-order face unknowns -> order-k unknowns (injection of the m = 0
    normal, t1 and t2 coefficients)."""
    nf = (k + 1) * (k + 2) // 2
    dpf = 3 * nf
    rows, cols = [], []
    for i in range(n_int):
        rows += [i * dpf, i * dpf + nf, i * dpf + 2 * nf]
        cols += [3 * i, 3 * i + 1, 3 * i + 2]
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n_int * dpf, 3 * n_int))


class MGhp3D(MGhp):
    """Algorithm 2 on a tetrahedral mesh: edge-patch relaxation of order k around MG_h."""

    def __init__(self, hdg_k: HDG3D, mgh: MGh3D, m_p: int = 1, m_h: int = 1, q: int = 1,
                 smoother: str = "gs", damping: float = 0.5, additive: bool = False):
        self.hdg = hdg_k
        self.A = hdg_k.matrix(with_al=True).tocsr()
        self.k = hdg_k.k
        self.mgh = mgh
        self.m_p, self.m_h, self.q = m_p, m_h, q
        self.additive = additive
        if self.k > 0:
            self.gs = make_smoother(self.A, edge_patches(hdg_k.topo, hdg_k.dpf), smoother, damping)
            self.Pi = inclusion_matrix_3d(hdg_k.topo.n_interior, self.k)


def build_hpmg_3d(topos: List[Topology3D], parents: List[np.ndarray], k: int, nu: float, beta: float,
                  gamma: float, m_p: int = 1, m_h: int = 1, q: int = 1, growth: int = 2,
                  hdg_k: Optional[HDG3D] = None, smoother: str = "gs", damping: float = 0.5,
                  additive: bool = False) -> MGhp3D:
    """hp-multigrid on the tetrahedral hierarchy topos[0] (coarsest) .. topos[-1] (finest)."""
    levels = [Level3D(HDG3D(t, 0, nu=nu, beta=beta, gamma=gamma), smoother, damping) for t in topos]
    mgh = MGh3D(levels, parents, growth=growth)
    if hdg_k is None:
        hdg_k = HDG3D(topos[-1], k, nu=nu, beta=beta, gamma=gamma)
    return MGhp3D(hdg_k, mgh, m_p=m_p, m_h=m_h, q=q, smoother=smoother, damping=damping, additive=additive)
