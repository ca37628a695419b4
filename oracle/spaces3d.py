"""Finite element spaces on one tetrahedron in physical coordinates (oracle).

TEST INFRASTRUCTURE ONLY.  As in 2D, everything is built directly on the physical
cell (no reference element, no Piola map).

Spaces (Section 2, d = 3):
* P^k(K): monomials in xi = (x - c)/h, c the centroid, h = (6|K|)^(1/3).
* RT_k(K) = [P^k]^3 ⊕ x P~^k, spanned by the vector monomials m e_a (m ∈ P^k,
  a = 1, 2, 3) and xi·h (h ∈ P~^k homogeneous of degree k); the spanning set is a
  basis ((k+1)(k+2)(k+4)/2 functions).  Its basis is dual to the degrees of freedom
      face f, m < (k+1)(k+2)/2:  ∫_F (v · n_F) ℓ_m dS,
      interior:                   ∫_K v · e_a xi^r,  a = 1, 2, 3,  r ∈ P^{k-1}.
* Face basis ℓ_m: the L2(F)-orthonormal basis obtained by Gram–Schmidt from the
  monomials λ_b^i λ_c^j (i + j <= k, by total degree then j) in the barycentric
  coordinates of the face's vertices x_b, x_c (sorted global order a < b < c).
  The tangential skeleton unknown on F is Σ_m (c1_m t1 + c2_m t2) ℓ_m.
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np

from .quadrature import face_points, tetrahedron_points


@lru_cache(maxsize=None)
def exponents3(deg: int):
    """Monomial exponents (a, b, c), a + b + c <= deg, by total degree."""
    out = []
    for n in range(deg + 1):
        for c in range(n + 1):
            for b in range(n - c + 1):
                out.append((n - b - c, b, c))
    return tuple(out)


@lru_cache(maxsize=None)
def homogeneous_exponents3(deg: int):
    return tuple(e for e in exponents3(deg) if sum(e) == deg)


@lru_cache(maxsize=None)
def face_exponents(k: int):
    """Exponents (i, j) of λ_b^i λ_c^j, i + j <= k, by total degree then j."""
    return tuple((n - j, j) for n in range(k + 1) for j in range(n + 1))


def n_face(k: int) -> int:
    return (k + 1) * (k + 2) // 2


def face_mono(ref, k):
    """Face monomials λ_b^i λ_c^j at reference face coordinates (λ_b, λ_c) = ref."""
    return np.stack([ref[:, 0] ** i * ref[:, 1] ** j for i, j in face_exponents(k)], axis=1)


def face_data(Xf: np.ndarray, k: int) -> dict:
    """Frame and scalar basis of the face with vertices Xf (3,3) in sorted global order:
    area, n_F, t1, t2 and `orth`, the coefficients of ℓ_m over the face monomials
    (Gram–Schmidt by the Cholesky factor of their Gram matrix)."""
    xa, xb, xc = Xf
    cr = np.cross(xb - xa, xc - xa)
    nF = cr / np.linalg.norm(cr)
    t1 = (xb - xa) / np.linalg.norm(xb - xa)
    _, ref, w = face_points(Xf, k + 2)
    Mo = face_mono(ref, k)
    G = (Mo * w[:, None]).T @ Mo
    return dict(Xf=np.asarray(Xf, dtype=float), area=0.5 * float(np.linalg.norm(cr)), nF=nF, t1=t1,
                t2=np.cross(nF, t1), orth=np.linalg.inv(np.linalg.cholesky(G)).T)


class Element3:
    """Geometry, orientation and bases of one tetrahedron.

    X: (4,3) vertex coordinates in the cell's local order; gv: (4,) global vertex
    ids (they fix the face frames and bases); k: polynomial order.
    """

    def __init__(self, X: np.ndarray, gv, k: int):
        self.X = np.asarray(X, dtype=np.float64)
        self.gv = [int(v) for v in gv]
        self.k = k
        J = np.stack([self.X[1] - self.X[0], self.X[2] - self.X[0], self.X[3] - self.X[0]], axis=1)
        self.vol = abs(np.linalg.det(J)) / 6.0
        self.area = self.vol                      # the cell measure |K| (name shared with 2D)
        self.c = self.X.mean(axis=0)
        self.h = (6.0 * self.vol) ** (1.0 / 3.0)
        self.nf = n_face(k)
        self.facets = []
        for f in range(4):
            loc = sorted((i for i in range(4) if i != f), key=lambda i: self.gv[i])
            fd = face_data(np.stack([self.X[i] for i in loc]), k)
            fd["sigma"] = 1.0 if fd["nF"] @ (fd["Xf"][0] - self.X[f]) > 0 else -1.0
            fd["nK"] = fd["sigma"] * fd["nF"]
            self.facets.append(fd)
        self._build_rt()

    # ---------------------------------------------------------------- monomials
    def xi(self, x):
        return (np.asarray(x) - self.c) / self.h

    def mono(self, x, deg):
        z = self.xi(x)
        return np.stack([z[:, 0] ** a * z[:, 1] ** b * z[:, 2] ** c for a, b, c in exponents3(deg)], axis=1)

    def mono_grad(self, x, deg):
        """Physical gradients (n, nm, 3) of the monomials of degree <= deg."""
        z = self.xi(x)
        out = np.zeros((z.shape[0], len(exponents3(deg)), 3))
        for i, e in enumerate(exponents3(deg)):
            for d in range(3):
                if e[d] > 0:
                    ee = list(e)
                    ee[d] -= 1
                    out[:, i, d] = e[d] * z[:, 0] ** ee[0] * z[:, 1] ** ee[1] * z[:, 2] ** ee[2] / self.h
        return out

    # ---------------------------------------------------------------- face basis
    def face_basis_ref(self, f, ref):
        """(n, nf) values of ℓ_m at reference face coordinates."""
        return face_mono(ref, self.k) @ self.facets[f]["orth"]

    def face_quad(self, f, n):
        """Quadrature on local face f: (physical points, ℓ values (n, nf), weights)."""
        fd = self.facets[f]
        x, ref, w = face_points(fd["Xf"], n)
        return x, self.face_basis_ref(f, ref), w

    # ---------------------------------------------------------------- RT_k
    def _span_coeffs(self):
        k = self.k
        E = exponents3(k + 1)
        idx = {e: i for i, e in enumerate(E)}
        rows = []
        for e in exponents3(k):
            for a in range(3):
                v = np.zeros((3, len(E)))
                v[a, idx[e]] = 1.0
                rows.append(v)
        for e in homogeneous_exponents3(k):
            v = np.zeros((3, len(E)))
            for a in range(3):
                ee = list(e)
                ee[a] += 1
                v[a, idx[tuple(ee)]] = 1.0
            rows.append(v)
        return np.asarray(rows)          # (n_span, 3, nm)

    def _build_rt(self):
        k = self.k
        S = self._span_coeffs()
        self.n_rt = S.shape[0]
        dof_rows = []
        for f in range(4):
            fd = self.facets[f]
            x, lm, w = self.face_quad(f, k + 3)
            vals = np.einsum("qm,jcm->qjc", self.mono(x, k + 1), S)
            vn = vals @ fd["nF"]
            for m in range(self.nf):
                dof_rows.append((w * lm[:, m]) @ vn)
        if k >= 1:
            xq, wq = tetrahedron_points(self.X, k + 2)
            vals = np.einsum("qm,jcm->qjc", self.mono(xq, k + 1), S)
            P = self.mono(xq, k - 1)
            for a in range(3):
                for r in range(P.shape[1]):
                    dof_rows.append((wq * P[:, r]) @ vals[:, :, a])
        V = np.asarray(dof_rows)
        assert V.shape[0] == V.shape[1] == self.n_rt
        self.rt_coeff = np.einsum("jcm,ji->icm", S, np.linalg.inv(V))  # (n_rt, 3, nm)
        self.n_rt_facet = 4 * self.nf

    def rt_values(self, x):
        return np.einsum("qm,icm->qic", self.mono(x, self.k + 1), self.rt_coeff)

    def rt_grads(self, x):
        """(n, n_rt, 3, 3) physical gradients, [q, i, comp, deriv]."""
        return np.einsum("qmd,icm->qicd", self.mono_grad(x, self.k + 1), self.rt_coeff)

    def rt_div(self, x):
        g = self.rt_grads(x)
        return g[:, :, 0, 0] + g[:, :, 1, 1] + g[:, :, 2, 2]
