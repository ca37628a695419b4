"""Finite element spaces on one triangle in physical coordinates (oracle).

TEST INFRASTRUCTURE ONLY.  Everything is built directly on the physical cell
(no reference element, no Piola map), which is a different route from the
CUDA library's reference-tensor construction.

Spaces (Section 2):
* P^k(K): monomials in xi = (x - c)/h, c the centroid, h = sqrt(2|K|).
* RT_k(K) = [P^k]^2 ⊕ x P~^k (P~^k homogeneous of degree k), spanned by the
  vector monomials (m, 0), (0, m) for m ∈ P^k and (xi h, eta h) for h ∈ P~^k.
  Its basis is dual to the degrees of freedom
      facet f, m = 0..k:  ∫_F (v · n_F) ℓ_m ds,
      interior:           ∫_K v · e_a xi^r,  a = 1, 2,  r ∈ P^{k-1},
  so a function is in the global (facet) part exactly when its interior
  moments vanish.  The skeleton unknowns of the scheme are these facet
  moments (normal trace) and the Legendre coefficients of the tangential
  facet unknown.
* Facet basis: ℓ_m(x) = sqrt(2m+1) P_m(2s-1) / sqrt(|F|), s ∈ [0,1] the
  facet parameter running from the lower to the higher global vertex id; the
  ℓ_m are L2-orthonormal on F.
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg

from .quadrature import gauss_legendre_01, triangle_points


@lru_cache(maxsize=None)
def exponents(deg: int):
    """Monomial exponents (a, b), a + b <= deg, ordered by total degree."""
    return tuple((n - b, b) for n in range(deg + 1) for b in range(n + 1))


@lru_cache(maxsize=None)
def homogeneous_exponents(deg: int):
    return tuple((deg - b, b) for b in range(deg + 1))


def legendre01(m: int, s: np.ndarray) -> np.ndarray:
    """sqrt(2m+1) P_m(2s-1): orthonormal Legendre polynomial on [0,1]."""
    c = np.zeros(m + 1)
    c[m] = 1.0
    return np.sqrt(2 * m + 1) * npleg.legval(2 * s - 1, c)


class Element:
    """Geometry, orientation and bases of one cell.

    X: (3,2) vertex coordinates in the cell's local order; gv: (3,) global
    vertex ids (they fix the facet orientations); k: polynomial order.
    """

    def __init__(self, X: np.ndarray, gv, k: int):
        self.X = np.asarray(X, dtype=np.float64)
        self.gv = [int(v) for v in gv]
        self.k = k
        J = np.stack([self.X[1] - self.X[0], self.X[2] - self.X[0]], axis=1)
        self.area = 0.5 * abs(np.linalg.det(J))
        self.c = self.X.mean(axis=0)
        self.h = np.sqrt(2.0 * self.area)
        self.facets = []
        for f in range(3):
            a, b = [i for i in range(3) if i != f]
            if self.gv[a] < self.gv[b]:
                lo, hi = a, b
            else:
                lo, hi = b, a
            xl, xh = self.X[lo], self.X[hi]
            d = xh - xl
            L = float(np.hypot(d[0], d[1]))
            t = d / L
            nF = np.array([t[1], -t[0]])
            mid = 0.5 * (xl + xh)
            sigma = 1.0 if nF @ (mid - self.X[f]) > 0 else -1.0
            self.facets.append(dict(xl=xl, xh=xh, L=L, t=t, nF=nF, sigma=sigma,
                                    nK=sigma * nF))
        self._build_rt()

    # ---------------------------------------------------------------- monomials
    def xi(self, x):
        return (np.asarray(x) - self.c) / self.h

    def mono(self, x, deg):
        """Values (n, nm) of the monomials of degree <= deg."""
        z = self.xi(x)
        return np.stack([z[:, 0] ** a * z[:, 1] ** b for a, b in exponents(deg)], axis=1)

    def mono_grad(self, x, deg):
        """Physical gradients (n, nm, 2) of the monomials of degree <= deg."""
        z = self.xi(x)
        out = np.zeros((z.shape[0], len(exponents(deg)), 2))
        for i, (a, b) in enumerate(exponents(deg)):
            if a > 0:
                out[:, i, 0] = a * z[:, 0] ** (a - 1) * z[:, 1] ** b / self.h
            if b > 0:
                out[:, i, 1] = b * z[:, 0] ** a * z[:, 1] ** (b - 1) / self.h
        return out

    # ---------------------------------------------------------------- RT_k
    def _span_coeffs(self):
        """Spanning set of RT_k as coefficients over monomials of degree <= k+1."""
        k = self.k
        E = exponents(k + 1)
        idx = {e: i for i, e in enumerate(E)}
        rows = []
        for e in exponents(k):
            v = np.zeros((2, len(E)))
            v[0, idx[e]] = 1.0
            rows.append(v)
            v = np.zeros((2, len(E)))
            v[1, idx[e]] = 1.0
            rows.append(v)
        for a, b in homogeneous_exponents(k):
            v = np.zeros((2, len(E)))
            v[0, idx[(a + 1, b)]] = 1.0
            v[1, idx[(a, b + 1)]] = 1.0
            rows.append(v)
        return np.asarray(rows)          # (n_span, 2, nm)

    def _build_rt(self):
        k = self.k
        S = self._span_coeffs()
        self.n_rt = S.shape[0]
        nq = k + 3
        dof_rows = []
        # facet normal moments against ℓ_m (global orientation)
        for f in range(3):
            fd = self.facets[f]
            s, w = gauss_legendre_01(nq)
            xq = fd["xl"][None, :] + s[:, None] * (fd["xh"] - fd["xl"])[None, :]
            vals = np.einsum("qm,jcm->qjc", self.mono(xq, k + 1), S)
            vn = vals @ fd["nF"]                        # (q, n_span)
            for m in range(k + 1):
                lm = legendre01(m, s) / np.sqrt(fd["L"])
                dof_rows.append((w * fd["L"] * lm) @ vn)
        # interior moments against e_a xi^r, r ∈ P^{k-1}
        if k >= 1:
            xq, wq = triangle_points(self.X, k + 2)
            vals = np.einsum("qm,jcm->qjc", self.mono(xq, k + 1), S)
            P = self.mono(xq, k - 1)
            for a in range(2):
                for r in range(P.shape[1]):
                    dof_rows.append((wq * P[:, r]) @ vals[:, :, a])
        V = np.asarray(dof_rows)
        self.rt_coeff = np.einsum("jcm,ji->icm", S, np.linalg.inv(V))  # (n_rt, 2, nm)
        self.n_rt_facet = 3 * (k + 1)

    def rt_values(self, x):
        """(n, n_rt, 2) values of the dual RT basis."""
        return np.einsum("qm,icm->qic", self.mono(x, self.k + 1), self.rt_coeff)

    def rt_grads(self, x):
        """(n, n_rt, 2, 2) physical gradients, [q, i, comp, deriv]."""
        return np.einsum("qmd,icm->qicd", self.mono_grad(x, self.k + 1), self.rt_coeff)

    def rt_div(self, x):
        g = self.rt_grads(x)
        return g[:, :, 0, 0] + g[:, :, 1, 1]

    def facet_legendre(self, f, s):
        """(n, k+1) values of ℓ_m on local facet f at global parameters s."""
        L = self.facets[f]["L"]
        return np.stack([legendre01(m, s) for m in range(self.k + 1)], axis=1) / np.sqrt(L)

    def facet_points(self, f, n):
        """Gauss–Legendre points (global parameter s, physical x, weights·|F|)."""
        fd = self.facets[f]
        s, w = gauss_legendre_01(n)
        x = fd["xl"][None, :] + s[:, None] * (fd["xh"] - fd["xl"])[None, :]
        return s, x, w * fd["L"]
