"""Quadrature rules (oracle; test infrastructure only).

Triangle rules are collapsed (Duffy) tensor rules: on the reference triangle
{xi, eta >= 0, xi + eta <= 1} with xi = (1+a)(1-b)/4, eta = (1+b)/2 the
Jacobian (1-b)/8 is absorbed by Gauss–Jacobi(alpha=1, beta=0) nodes in b, and
Gauss–Legendre nodes are used in a.  n nodes per direction integrate every
polynomial of total degree <= 2n-1 exactly.  The 1D nodes come from SciPy's
orthogonal-polynomial routines (library primitives).
"""

from functools import lru_cache

import numpy as np
from scipy.special import roots_jacobi, roots_legendre


@lru_cache(maxsize=None)
def gauss_legendre_01(n: int):
    """n-point Gauss–Legendre rule on [0, 1]: (points (n,), weights (n,))."""
    x, w = roots_legendre(n)
    return 0.5 * (x + 1.0), 0.5 * w


@lru_cache(maxsize=None)
def triangle_rule(n: int):
    """Collapsed rule on the reference triangle: (points (n²,2), weights (n²,))."""
    a, wa = roots_legendre(n)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    xi = (1 + A) * (1 - B) / 4
    eta = (1 + B) / 2
    pts = np.stack([xi.ravel(), eta.ravel()], axis=1)
    w = (WA * WB).ravel() / 8.0
    return pts, w


def triangle_points(X: np.ndarray, n: int):
    """Physical rule on triangle with vertices X (3,2): (points, weights)."""
    ref, w = triangle_rule(n)
    J = np.stack([X[1] - X[0], X[2] - X[0]], axis=1)
    det = abs(np.linalg.det(J))
    return X[0] + ref @ J.T, w * det


@lru_cache(maxsize=None)
def tetrahedron_rule(n: int):
    """Collapsed (conical product) rule on the reference tetrahedron
    {xi, eta, zeta >= 0, xi + eta + zeta <= 1}: xi = (1+a)(1-b)(1-c)/8,
    eta = (1+b)(1-c)/4, zeta = (1+c)/2 with Jacobian (1-b)(1-c)²/64, absorbed by
    Gauss–Jacobi(1, 0) nodes in b and Gauss–Jacobi(2, 0) nodes in c; Gauss–Legendre
    in a.  Exact for total degree <= 2n-1.  Returns (points (n³, 3), weights (n³,)),
    sum of weights 1/6."""
    a, wa = roots_legendre(n)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    c, wc = roots_jacobi(n, 2.0, 0.0)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    W = np.einsum("i,j,k->ijk", wa, wb, wc)
    xi = (1 + A) * (1 - B) * (1 - C) / 8
    eta = (1 + B) * (1 - C) / 4
    zeta = (1 + C) / 2
    pts = np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], axis=1)
    return pts, W.ravel() / 64.0


def tetrahedron_points(X: np.ndarray, n: int):
    """Physical rule on the tetrahedron with vertices X (4,3): (points, weights)."""
    ref, w = tetrahedron_rule(n)
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    return X[0] + ref @ J.T, w * abs(np.linalg.det(J))


def face_points(Xf: np.ndarray, n: int):
    """Physical rule on a triangle embedded in 3D with vertices Xf (3,3): (points,
    reference coordinates (n², 2) along the edges Xf[1]-Xf[0], Xf[2]-Xf[0], weights)."""
    ref, w = triangle_rule(n)
    E = np.stack([Xf[1] - Xf[0], Xf[2] - Xf[0]], axis=1)          # (3, 2)
    area2 = np.linalg.norm(np.cross(E[:, 0], E[:, 1]))
    return Xf[0] + ref @ E.T, ref, w * area2
