"""Flexible GMRES and the augmented-Lagrangian Uzawa iteration (oracle).

TEST INFRASTRUCTURE ONLY.

* FGMRES (right preconditioning, preconditioner allowed to vary): Arnoldi
  with classical Gram–Schmidt applied twice, Givens rotations on the
  Hessenberg matrix, stop when the Euclidean norm of the residual vector
  is <= an absolute target (the caller derives it from the relative 1e-8 /
  absolute 1e-10 settings of Section 5), restart length 30.  The Krylov
  method is GMRES by default because the mixed-precision preconditioner is
  not exactly linear; the paper uses PCG for Stokes (Section 5), available
  as ``pcg`` (symmetric problems and preconditioners only).
* Uzawa (eq. stOpEq-ALU): p⁰ = 0;  A^ε u⁽ⁿ⁾ = F − B*p⁽ⁿ⁻¹⁾;
  p⁽ⁿ⁾ = p⁽ⁿ⁻¹⁾ − ε⁻¹ div u⁽ⁿ⁾ on every cell.  With the flux matrix D
  ((D u)_K = ∫_{∂K} u·n) this is  A^ε u = F + Dᵀp,  p_K ← p_K − ε⁻¹ (Du)_K/|K|.
  The update is written with div u: with B as defined in eq. stOptForm
  ([Bu, q] = −(div u, q)) the printed sign would make the iteration diverge;
  the form above is the one whose error contracts by ε/(ε+μ0) per step
  (Lemma 3.1).  The inner solves are warm-started from the previous u and,
  as in Section 5, stop at relative 1e-8 / absolute 1e-10, but never below
  floor_rel·‖F‖ (default 1e-10; Remark 3.1: much smaller residuals are
  round-off at large ε⁻¹):
  ‖g − A^ε u‖ <= max(rtol·‖g − A^ε u_start‖, floor_rel·‖F‖, atol).
  An inner solve that stagnates on round-off (see ``fgmres``) raises the floor
  to twice its final residual for the later Uzawa steps.
  The outer loop stops once the pressure error estimate of a linearly
  converging iteration, ρ/(1−ρ)·‖p⁽ⁿ⁾ − p⁽ⁿ⁻¹⁾‖ with ρ the observed ratio of
  successive updates (Lemma 3.1 gives ρ = ε/(ε+μ0)), is <= uzawa_tol·‖p⁽ⁿ⁾‖
  in L2(Ω), or when an inner solve makes no progress.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import scipy.linalg as sla


def fgmres(A, b, x0, M: Callable, rtol: float = 1e-8, atol: float = 1e-10,
           restart: int = 30, max_it: int = 1000, info: Optional[dict] = None):
    """Solve A x = b to ‖r‖ <= max(rtol‖r0‖, atol).

    Returns (x, iterations, final residual norm, history of residual norms).  A
    restart cycle that ends because the Givens estimate met the tolerance while the
    true residual did not shows round-off in the residual (Remark 3.1); when the
    next such cycle cuts the true residual by less than half the solve stops as
    stagnated (info["stagnated"] = True when a dict is passed).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    total = 0
    hist = []
    tol = None
    beta_prev = None
    est_reached = False
    if info is not None:
        info["stagnated"] = False
    while True:
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        if tol is None:
            tol = max(rtol * beta, atol)
        hist.append(beta)
        if beta <= tol or total >= max_it:
            return x, total, beta, hist
        if est_reached and beta_prev is not None and beta > 0.5 * beta_prev:
            if info is not None:
                info["stagnated"] = True
            return x, total, beta, hist
        beta_prev = beta
        est_reached = False
        n = b.shape[0]
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(restart):
            Z[j] = M(V[j])
            w = A @ Z[j]
            h1 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h1
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h1 + h2
            hn = float(np.linalg.norm(w))
            col = np.zeros(restart + 1)
            col[:j + 1] = h
            col[j + 1] = hn
            for i in range(j):
                a, bb = col[i], col[i + 1]
                col[i] = cs[i] * a + sn[i] * bb
                col[i + 1] = -sn[i] * a + cs[i] * bb
            den = float(np.hypot(col[j], col[j + 1]))
            cs[j] = col[j] / den
            sn[j] = col[j + 1] / den
            col[j] = den
            col[j + 1] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            H[:, j] = col
            total += 1
            j_end = j
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol:
                est_reached = True
            if abs(g[j + 1]) <= tol or total >= max_it or hn == 0.0:
                break
            V[j + 1] = w / hn
        m = j_end + 1
        y = sla.solve_triangular(H[:m, :m], g[:m])
        x = x + Z[:m].T @ y


def pcg(A, b, x0, M: Callable, rtol: float = 1e-8, atol: float = 1e-10, max_it: int = 1000):
    """Preconditioned conjugate gradients (the paper's Krylov method for the generalized
    Stokes problem, Section 5) for symmetric positive definite A and a symmetric
    preconditioner M: stop when the recursively updated residual has
    ‖r‖ <= max(rtol‖r0‖, atol), the same norm and targets as ``fgmres``.

    Returns (x, iterations, final residual norm, history of residual norms).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    beta0 = float(np.linalg.norm(r))
    tol = max(rtol * beta0, atol)
    hist = [beta0]
    if beta0 <= tol:
        return x, 0, beta0, hist
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    its = 0
    rn = beta0
    while its < max_it:
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        its += 1
        rn = float(np.linalg.norm(r))
        hist.append(rn)
        if rn <= tol:
            break
        z = M(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, its, rn, hist


@dataclass
class UzawaResult:
    u: np.ndarray
    p: np.ndarray
    krylov_its: List[int] = field(default_factory=list)
    res_mom: float = 0.0
    res_div: float = 0.0
    dp_rel: float = 0.0
    normF: float = 0.0
    div_l2: float = 0.0      # ‖div u_h‖_L2: div u_h is the cell flux sum over |K| on every cell
    res_floor: float = 0.0   # final inner floor (raised on stagnation)


def uzawa(Aeps, D, area, eps_inv, F, M: Callable, rtol: float = 1e-8, atol: float = 1e-10,
          restart: int = 30, max_it: int = 1000, max_uzawa: int = 200,
          uzawa_tol: float = 1e-8, floor_rel: float = 1e-10, u0=None,
          krylov: str = "fgmres", bflux=None) -> UzawaResult:
    """Augmented-Lagrangian Uzawa with FGMRES (or, krylov="pcg", PCG) inner solves
    (eq. stOpEq-ALU).  bflux: per-cell fluxes of inhomogeneous Dirichlet data, added to
    D u in the pressure update (None = homogeneous data)."""
    normF = float(np.linalg.norm(F))
    u = np.zeros_like(F) if u0 is None else np.array(u0, copy=True)
    p = np.zeros(D.shape[0])
    res = UzawaResult(u=u, p=p, normF=normF)
    floor = max(floor_rel * normF, atol)
    ndp_prev = None
    for n in range(max_uzawa):
        g = F + D.T @ p
        fi = {"stagnated": False}
        if krylov == "pcg":
            u, its, rn, _ = pcg(Aeps, g, u, M, rtol=rtol, atol=floor, max_it=max_it)
        else:
            u, its, rn, _ = fgmres(Aeps, g, u, M, rtol=rtol, atol=floor, restart=restart,
                                   max_it=max_it, info=fi)
        # an inner solve that stagnated on round-off raises the floor of the later ones
        if fi["stagnated"]:
            floor = max(floor, 2.0 * rn)
        res.res_floor = floor
        du = D @ u if bflux is None else D @ u + bflux
        res.div_l2 = float(np.sqrt(np.sum(du ** 2 / area)))
        dp = eps_inv * du / area
        p = p - dp
        res.krylov_its.append(its)
        res.res_mom = rn
        res.res_div = float(np.linalg.norm(du))
        ndp = float(np.sqrt(area @ dp ** 2))
        npn = float(np.sqrt(area @ p ** 2))
        res.dp_rel = ndp / npn if npn > 0 else 0.0
        if ndp <= atol or (n > 0 and its == 0):
            break
        if ndp_prev is not None:
            rho = min(ndp / ndp_prev, 0.99)
            if rho / (1.0 - rho) * ndp <= uzawa_tol * npn:
                break
        ndp_prev = ndp
    res.u, res.p = u, p
    return res
