"""Manufactured solutions of the generalized Stokes problem and forcing samples.

The model problem is -div(nu grad u) + beta u + grad p = f, div u = 0 in
Omega = (0,1)^2, u = 0 on the boundary (Section 3.1, eq. stModel).  Each
solution below is given in closed form together with its gradient and its
Laplacian, so that the forcing f = -nu Δu + beta u + grad p is exact.

* ``curl_bubble_2d``: u = curl psi = (d psi/dy, -d psi/dx) with
  psi = sin²(pi x) sin²(pi y) and p = sin(2 pi x) cos(2 pi y).
* ``polynomial_2d``: the paper's 2D convergence-check solution
  (Section 5.1), u = (-g(x) g'(y), g'(x) g(y)) with g(t) = t²(t-1)² and
  p = x(1-x)(1-y) - 1/12.

Forcing enters the library as values of a vector polynomial of degree k+1 on
each cell, sampled at the cell's degree-(k+1) lattice points (see
``lattice_points_2d``).  Sampling the exact f there defines the discrete
forcing f_h ∈ [P^{k+1}(K)]^2 element by element.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

PI = np.pi


@dataclass
class Solution2D:
    """Exact velocity, velocity gradient, pressure and Laplacian at points."""
    u: Callable[[np.ndarray], np.ndarray]        # (n,2) -> (n,2)
    grad_u: Callable[[np.ndarray], np.ndarray]   # (n,2) -> (n,2,2), [i,j] = d u_i / d x_j
    lap_u: Callable[[np.ndarray], np.ndarray]    # (n,2) -> (n,2)
    p: Callable[[np.ndarray], np.ndarray]        # (n,2) -> (n,)
    grad_p: Callable[[np.ndarray], np.ndarray]   # (n,2) -> (n,2)

    def forcing(self, nu: float, beta: float,
                conv: Optional[Callable[[np.ndarray], np.ndarray]] = None
                ) -> Callable[[np.ndarray], np.ndarray]:
        """f = -nu Δu + beta u + grad p (+ (b·grad) u when a convecting field b is given)."""
        def f(x):
            val = -nu * self.lap_u(x) + beta * self.u(x) + self.grad_p(x)
            if conv is not None:
                b = conv(x)
                val = val + np.einsum("nij,nj->ni", self.grad_u(x), b)
            return val
        return f


def curl_bubble_2d() -> Solution2D:
    s = lambda t: np.sin(PI * t) ** 2
    s1 = lambda t: PI * np.sin(2 * PI * t)
    s2 = lambda t: 2 * PI ** 2 * np.cos(2 * PI * t)
    s3 = lambda t: -4 * PI ** 3 * np.sin(2 * PI * t)

    def u(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([s(X) * s1(Y), -s1(X) * s(Y)], axis=1)

    def grad_u(x):
        X, Y = x[:, 0], x[:, 1]
        g = np.empty((x.shape[0], 2, 2))
        g[:, 0, 0] = s1(X) * s1(Y)
        g[:, 0, 1] = s(X) * s2(Y)
        g[:, 1, 0] = -s2(X) * s(Y)
        g[:, 1, 1] = -s1(X) * s1(Y)
        return g

    def lap_u(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([s2(X) * s1(Y) + s(X) * s3(Y),
                         -s3(X) * s(Y) - s1(X) * s2(Y)], axis=1)

    def p(x):
        return np.sin(2 * PI * x[:, 0]) * np.cos(2 * PI * x[:, 1])

    def grad_p(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([2 * PI * np.cos(2 * PI * X) * np.cos(2 * PI * Y),
                         -2 * PI * np.sin(2 * PI * X) * np.sin(2 * PI * Y)], axis=1)

    return Solution2D(u, grad_u, lap_u, p, grad_p)


def polynomial_2d() -> Solution2D:
    g = lambda t: t ** 2 * (t - 1) ** 2
    g1 = lambda t: 4 * t ** 3 - 6 * t ** 2 + 2 * t
    g2 = lambda t: 12 * t ** 2 - 12 * t + 2
    g3 = lambda t: 24 * t - 12

    def u(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([-g(X) * g1(Y), g1(X) * g(Y)], axis=1)

    def grad_u(x):
        X, Y = x[:, 0], x[:, 1]
        G = np.empty((x.shape[0], 2, 2))
        G[:, 0, 0] = -g1(X) * g1(Y)
        G[:, 0, 1] = -g(X) * g2(Y)
        G[:, 1, 0] = g2(X) * g(Y)
        G[:, 1, 1] = g1(X) * g1(Y)
        return G

    def lap_u(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([-g2(X) * g1(Y) - g(X) * g3(Y),
                         g3(X) * g(Y) + g1(X) * g2(Y)], axis=1)

    def p(x):
        X, Y = x[:, 0], x[:, 1]
        return X * (1 - X) * (1 - Y) - 1.0 / 12.0

    def grad_p(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([(1 - 2 * X) * (1 - Y), -X * (1 - X)], axis=1)

    return Solution2D(u, grad_u, lap_u, p, grad_p)


def n_lattice_2d(q: int) -> int:
    return (q + 1) * (q + 2) // 2


def lattice_barycentric_2d(q: int) -> np.ndarray:
    """(n, 3) barycentric coordinates of the degree-q lattice of a triangle.

    Order: for a2 = 0..q, for a1 = 0..q-a2: (lambda1, lambda2) = (a1/q, a2/q),
    lambda0 = 1 - lambda1 - lambda2.  For q = 0 the single point is the centroid.
    """
    if q == 0:
        return np.array([[1 / 3, 1 / 3, 1 / 3]])
    pts = []
    for a2 in range(q + 1):
        for a1 in range(q + 1 - a2):
            l1, l2 = a1 / q, a2 / q
            pts.append((1 - l1 - l2, l1, l2))
    return np.asarray(pts)


def lattice_points_2d(coords: np.ndarray, cells: np.ndarray, q: int) -> np.ndarray:
    """(n_cells, n_lattice, 2) physical lattice points of every cell."""
    lam = lattice_barycentric_2d(q)
    V = coords[cells]                      # (nc, 3, 2)
    return np.einsum("pv,cvd->cpd", lam, V)


def forcing_at_lattice(coords: np.ndarray, cells: np.ndarray, k: int,
                       f: Callable[[np.ndarray], np.ndarray]) -> np.ndarray:
    """Forcing samples (n_cells, n_lattice(k+1), d) at the degree-(k+1) lattice (d = 2 for
    triangles, 3 for tetrahedra)."""
    d = coords.shape[1]
    X = (lattice_points_2d if d == 2 else lattice_points_3d)(coords, cells, k + 1)
    nc, npt, _ = X.shape
    return f(X.reshape(-1, d)).reshape(nc, npt, d)


def n_lattice_3d(q: int) -> int:
    return (q + 1) * (q + 2) * (q + 3) // 6


def lattice_barycentric_3d(q: int) -> np.ndarray:
    """(n, 4) barycentric coordinates of the degree-q lattice of a tetrahedron.

    Order: for a3 = 0..q, for a2 = 0..q-a3, for a1 = 0..q-a2-a3:
    (lambda1, lambda2, lambda3) = (a1, a2, a3)/q, lambda0 = 1 - lambda1 - lambda2 - lambda3.
    For q = 0 the single point is the centroid.
    """
    if q == 0:
        return np.full((1, 4), 0.25)
    pts = []
    for a3 in range(q + 1):
        for a2 in range(q + 1 - a3):
            for a1 in range(q + 1 - a2 - a3):
                l1, l2, l3 = a1 / q, a2 / q, a3 / q
                pts.append((1 - l1 - l2 - l3, l1, l2, l3))
    return np.asarray(pts)


def lattice_points_3d(coords: np.ndarray, cells: np.ndarray, q: int) -> np.ndarray:
    """(n_cells, n_lattice, 3) physical lattice points of every tetrahedron."""
    lam = lattice_barycentric_3d(q)
    V = coords[cells]                      # (nc, 4, 3)
    return np.einsum("pv,cvd->cpd", lam, V)


def curl_bubble_3d() -> Solution2D:
    """The 3D manufactured solution: u = grad psi x (1, 1, 1) with
    psi = sin²(pi x) sin²(pi y) sin²(pi z) (divergence free, zero on the boundary of the
    unit cube) and p = sin(2 pi x) cos(2 pi y) sin(2 pi z) (mean free)."""
    s = lambda t: np.sin(PI * t) ** 2
    s1 = lambda t: PI * np.sin(2 * PI * t)
    s2 = lambda t: 2 * PI ** 2 * np.cos(2 * PI * t)
    s3 = lambda t: -4 * PI ** 3 * np.sin(2 * PI * t)
    D = (s, s1, s2, s3)

    def dpsi(x, a, b, c):
        """d^(a,b,c) psi at points x (a, b, c <= 3 derivatives per coordinate)."""
        return D[a](x[:, 0]) * D[b](x[:, 1]) * D[c](x[:, 2])

    def e(i):
        t = [0, 0, 0]
        t[i] += 1
        return t

    def grad_psi_d(x, extra):
        """(n, 3): component i = d_i psi differentiated further by the multi-index extra."""
        return np.stack([dpsi(x, *(np.array(e(i)) + np.array(extra))) for i in range(3)], axis=1)

    def from_grad(G):
        # u = grad psi x (1,1,1) = (psi_y - psi_z, psi_z - psi_x, psi_x - psi_y)
        return np.stack([G[:, 1] - G[:, 2], G[:, 2] - G[:, 0], G[:, 0] - G[:, 1]], axis=1)

    def u(x):
        return from_grad(grad_psi_d(x, (0, 0, 0)))

    def grad_u(x):
        g = np.empty((x.shape[0], 3, 3))
        for j in range(3):
            g[:, :, j] = from_grad(grad_psi_d(x, e(j)))
        return g

    def lap_u(x):
        return sum(from_grad(grad_psi_d(x, [2 * (i == j) for i in range(3)])) for j in range(3))

    def p(x):
        return np.sin(2 * PI * x[:, 0]) * np.cos(2 * PI * x[:, 1]) * np.sin(2 * PI * x[:, 2])

    def grad_p(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        sx, cx = np.sin(2 * PI * X), np.cos(2 * PI * X)
        sy, cy = np.sin(2 * PI * Y), np.cos(2 * PI * Y)
        sz, cz = np.sin(2 * PI * Z), np.cos(2 * PI * Z)
        return 2 * PI * np.stack([cx * cy * sz, -sx * sy * sz, sx * cy * cz], axis=1)

    return Solution2D(u, grad_u, lap_u, p, grad_p)


def gradient_field_2d(a: np.ndarray):
    """grad phi for phi = sum_{i+j<=deg} a[i,j] x^i y^j (a: (deg+1, deg+1)).

    Used to add an irrotational field to the forcing; returns (phi, grad phi).
    """
    deg = a.shape[0] - 1

    def phi(x):
        X, Y = x[:, 0], x[:, 1]
        out = np.zeros(x.shape[0])
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                out += a[i, j] * X ** i * Y ** j
        return out

    def grad(x):
        X, Y = x[:, 0], x[:, 1]
        gx = np.zeros(x.shape[0])
        gy = np.zeros(x.shape[0])
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                if i > 0:
                    gx += a[i, j] * i * X ** (i - 1) * Y ** j
                if j > 0:
                    gy += a[i, j] * j * X ** i * Y ** (j - 1)
        return np.stack([gx, gy], axis=1)

    return phi, grad


def seeded_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal test vector from numpy's PCG64 with the given seed."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)



def convecting_stream_2d(scale: float = 1.0):
    """(psi, b) with psi = c sin²(pi x) sin²(pi y) and b = curl psi = (d psi/dy, -d psi/dx).

    c is chosen so that max|b| = scale on the unit square.  b is divergence
    free and b·n = 0 on the boundary (psi vanishes there).
    """
    bub = curl_bubble_2d()
    g = np.linspace(0.0, 1.0, 801)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    c = scale / float(np.sqrt((bub.u(pts) ** 2).sum(axis=1)).max())

    def psi(x):
        return c * (np.sin(PI * x[:, 0]) * np.sin(PI * x[:, 1])) ** 2

    def b(x):
        return c * bub.u(x)

    return psi, b


def _lattice_lagrange_gradients(q: int) -> np.ndarray:
    """(n, n, 2): reference-triangle gradient of Lagrange basis function n' at lattice point n."""
    lam = lattice_barycentric_2d(q)
    xy = lam[:, 1:]                                   # reference coordinates (lambda1, lambda2)
    ex = [(d - b, b) for d in range(q + 1) for b in range(d + 1)]
    V = np.stack([xy[:, 0] ** a * xy[:, 1] ** b for a, b in ex], axis=1)
    Vx = np.stack([a * xy[:, 0] ** max(a - 1, 0) * xy[:, 1] ** b if a else 0 * xy[:, 0]
                   for a, b in ex], axis=1)
    Vy = np.stack([b * xy[:, 0] ** a * xy[:, 1] ** max(b - 1, 0) if b else 0 * xy[:, 0]
                   for a, b in ex], axis=1)
    Vi = np.linalg.inv(V)
    return np.stack([Vx @ Vi, Vy @ Vi], axis=2)


def curl_lattice_2d(coords: np.ndarray, cells: np.ndarray, q: int,
                    psi: Callable[[np.ndarray], np.ndarray]) -> np.ndarray:
    """(n_cells, n_lattice(q), 2): curl of the continuous degree-q Lagrange
    interpolant psi_h of psi, sampled at each cell's degree-q lattice.

    curl psi_h = (d psi_h/dy, -d psi_h/dx) is a piecewise polynomial of degree
    q-1 with single-valued normal component across cells and zero divergence,
    and it is tangential on the boundary wherever psi vanishes there: a
    divergence-free member of the Raviart–Thomas space RT_{q-1}.
    """
    X = lattice_points_2d(coords, cells, q)               # (nc, n, 2)
    nc, n, _ = X.shape
    vals = psi(X.reshape(-1, 2)).reshape(nc, n)
    D = _lattice_lagrange_gradients(q)                    # (n, n', 2) reference gradients
    gref = np.einsum("mnd,cn->cmd", D, vals)              # (nc, n, 2) reference gradient
    V = coords[cells]
    J = np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]], axis=2)   # (nc, 2, 2) columns = edges
    Jinv = np.linalg.inv(J)
    grad = np.einsum("cdi,cmd->cmi", Jinv, gref)          # J^{-T} ∇̂
    return np.stack([grad[..., 1], -grad[..., 0]], axis=2)


def fourier_forcing_2d(j: int, n_modes: int = 8, seed0: int = 20230312):
    """Seeded forcing number j of the many-right-hand-side workload:
    f_j = Σ_m a_m sin(2π(p_m x + q_m y) + θ_m) + ∇φ_j,
    φ_j = Σ_m b_m cos(2π(r_m x + s_m y) + η_m),
    a_m ~ N(0, I_2), b_m ~ N(0, 1), integer wavenumbers p, q, r, s in 1..8 and
    phases θ, η ~ U[0, 2π), all drawn from numpy.random.default_rng(seed0 + j)."""
    rng = np.random.default_rng(seed0 + j)
    a = rng.standard_normal((n_modes, 2))
    pq = rng.integers(1, 9, size=(n_modes, 2))
    th = rng.uniform(0.0, 2 * PI, n_modes)
    b = rng.standard_normal(n_modes)
    rs = rng.integers(1, 9, size=(n_modes, 2))
    eta = rng.uniform(0.0, 2 * PI, n_modes)

    def f(x, xp=np):
        """x: (n, 2) points; xp: the array module of x (numpy, or torch for device arrays)."""
        out = xp.zeros_like(x)
        for m in range(n_modes):
            arg = 2 * PI * (float(pq[m, 0]) * x[:, 0] + float(pq[m, 1]) * x[:, 1]) + float(th[m])
            s = xp.sin(arg)
            out[:, 0] += float(a[m, 0]) * s
            out[:, 1] += float(a[m, 1]) * s
            # ∇ of b cos(argp)
            argp = 2 * PI * (float(rs[m, 0]) * x[:, 0] + float(rs[m, 1]) * x[:, 1]) + float(eta[m])
            sp = (-2 * PI * float(b[m])) * xp.sin(argp)
            out[:, 0] += float(rs[m, 0]) * sp
            out[:, 1] += float(rs[m, 1]) * sp
        return out

    return f


def boundary_facets_2d(cells: np.ndarray) -> np.ndarray:
    """(n_boundary, 2) sorted global vertex pairs of the boundary facets in facet order
    (lexicographic in the sorted pair), the order of the Dirichlet data."""
    e = np.concatenate([cells[:, [1, 2]], cells[:, [0, 2]], cells[:, [0, 1]]])
    e.sort(axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    return uniq[cnt == 1]


def dirichlet_facet_data(coords: np.ndarray, cells: np.ndarray, k: int,
                         g: Callable[[np.ndarray], np.ndarray], nq: Optional[int] = None) -> np.ndarray:
    """Skeleton values (n_boundary, 2(k+1)) of boundary data g in the unknowns' layout: on a
    facet F from its lower to its higher global vertex (unit tangent t, normal
    n = (t_y, -t_x), parameter s from the lower vertex, l_m = sqrt(2m+1) P_m(2s-1)/sqrt|F|),
    the normal moments int_F (g.n) l_m ds for m = 0..k, then the tangential coefficients
    int_F (g.t) l_m ds, by Gauss-Legendre quadrature on each facet."""
    pairs = boundary_facets_2d(cells)
    nq = nq or (k + 6)
    z, w = np.polynomial.legendre.leggauss(nq)
    s, w = 0.5 * (z + 1), 0.5 * w
    X0, X1 = coords[pairs[:, 0]], coords[pairs[:, 1]]
    L = np.linalg.norm(X1 - X0, axis=1)
    t = (X1 - X0) / L[:, None]
    n = np.stack([t[:, 1], -t[:, 0]], axis=1)
    pts = X0[:, None, :] + s[None, :, None] * (X1 - X0)[:, None, :]
    gv = g(pts.reshape(-1, 2)).reshape(len(pairs), nq, 2)
    gn = np.einsum("fqd,fd->fq", gv, n)
    gt = np.einsum("fqd,fd->fq", gv, t)
    leg = np.stack([np.sqrt(2 * m + 1) * np.polynomial.legendre.legval(2 * s - 1, [0] * m + [1])
                    for m in range(k + 1)], axis=1)                       # (nq, k+1)
    # int_F v l_m ds = |F| int_0^1 v(s) sqrt(2m+1) P_m(2s-1) ds / sqrt|F|
    scale = np.sqrt(L)[:, None]
    return np.concatenate([scale * (gn * w) @ leg, scale * (gt * w) @ leg], axis=1)


def lid_velocity_2d(speed: float = 1.0) -> Callable[[np.ndarray], np.ndarray]:
    """Driven-lid boundary data of the cavity problem (Section 5.2 workloads): tangential
    velocity (speed, 0) on the top side y = 1, zero on the other sides."""
    def g(x):
        out = np.zeros_like(x)
        out[np.isclose(x[:, 1], 1.0), 0] = speed
        return out
    return g


def step_channel_velocity_2d() -> Callable[[np.ndarray], np.ndarray]:
    """Boundary data of the backward-facing-step stand-in (Section 5.3 workloads): a parabolic
    inflow (16 (y - 1/2)(1 - y), 0) on x = 0, 1/2 < y < 1, a parabolic outflow (2 y (1 - y), 0)
    on x = 4 carrying the same flux 1/3, and no-slip walls.  The paper's do-nothing outflow is
    replaced by this prescribed profile."""
    def g(x):
        out = np.zeros_like(x)
        inl = np.isclose(x[:, 0], 0.0) & (x[:, 1] > 0.5)
        out[inl, 0] = 16.0 * (x[inl, 1] - 0.5) * (1.0 - x[inl, 1])
        outl = np.isclose(x[:, 0], 4.0)
        out[outl, 0] = 2.0 * x[outl, 1] * (1.0 - x[outl, 1])
        return out
    return g
