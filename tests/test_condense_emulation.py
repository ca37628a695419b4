"""Host-side pin of the device condensation (no GPU).

The library's reference-element tables (exported by hdg_reference_tables) are
contracted with each cell's Jacobian exactly as the condensation kernel does
(Piola map, global facet scaling sqrt|F|·σ·sgn(det J)·o^m, closed-form flux
elimination, block Cholesky of the interior velocity / mean-free pressure
unknowns, AL term), here in NumPy, and compared with the oracle's condensed
matrices and loads, which are built along a different route (physical
coordinates, dense Schur complement of the full local system).  A mistake in
the tables or in the kernel's algebra shows up here before any GPU run.
"""
import numpy as np
import pytest

from workloads import unit_square, curl_bubble_2d
from oracle.hdg import HDG
from _util import topo_of, forcing, rel

FV = [(1, 2), (0, 2), (0, 1)]
FL = [np.sqrt(2.0), 1.0, 1.0]


def emulate_cell(X, gv, k, nu, beta, eps_inv, fn, T):
    npk, nrt, nf = (k + 1) * (k + 2) // 2, (k + 1) * (k + 3), k + 1
    nL, ng, nri, npo = 4 * npk, 6 * nf, k * (k + 1), npk - 1
    J = np.array([[X[1, 0] - X[0, 0], X[2, 0] - X[0, 0]], [X[1, 1] - X[0, 1], X[2, 1] - X[0, 1]]])
    det = np.linalg.det(J)
    sgn = 1.0 if det > 0 else -1.0
    Ji = np.linalg.inv(J)
    ln, nK, tF, sig, o = [], [], [], [], []
    for f, (a, b) in enumerate(FV):
        d = X[b] - X[a]
        L = np.hypot(*d)
        of = 1.0 if gv[a] < gv[b] else -1.0
        t = of * d / L
        n = np.array([t[1], -t[0]])
        s = 1.0 if n @ (0.5 * (X[a] + X[b]) - X[f]) > 0 else -1.0
        ln.append(L); nK.append(s * n); tF.append(t); sig.append(s); o.append(of)
    sc = np.ones(nrt)
    for f in range(3):
        for m in range(nf):
            sc[f * nf + m] = np.sqrt(ln[f]) * sig[f] * sgn * (o[f] if m % 2 else 1.0)
    C = np.zeros((nL, nrt + 3 * nf))
    for c in range(2):
        for e in range(2):
            rows = slice((2 * c + e) * npk, (2 * c + e + 1) * npk)
            vol = sgn * np.einsum("a,b,iabj->ji", J[c], Ji[:, e], T["R1"])
            bnd = np.zeros((npk, nrt))
            for f in range(3):
                P = J[c] - nK[f][c] * (nK[f] @ J)
                bnd += ln[f] / FL[f] / det * nK[f][e] * np.einsum("a,iaj->ji", P, T["R2"][f])
            C[rows, :nrt] = (vol - bnd) * sc[None, :]
            for f in range(3):
                om = np.array([o[f] ** m for m in range(nf)])
                C[rows, nrt + f * nf:nrt + (f + 1) * nf] = nK[f][e] * tF[f][c] * np.sqrt(ln[f]) * \
                    T["R3"][f] * om[None, :]
    Dm = sgn * T["R5"] * sc[:, None]
    JtF = fn.reshape(-1, 2) @ J                             # (n_lat, 2): (J^T F_n)_a
    Fl = sgn * np.einsum("na,ian->i", JtF, T["R6"]) * sc
    K = nu / abs(det) * C.T @ C
    M = np.einsum("ab,iajb->ij", J.T @ J, T["R4"])
    K[:nrt, :nrt] += beta / abs(det) * M * np.outer(sc, sc)
    gcol = []
    for f in range(3):
        gcol += [f * nf + m for m in range(nf)] + [nrt + f * nf + m for m in range(nf)]
    gcol = np.array(gcol)
    ii = np.arange(3 * nf, nrt)
    A = K[np.ix_(gcol, gcol)].copy()
    Fg = np.where(gcol < nrt, Fl[np.minimum(gcol, nrt - 1)], 0.0)
    if nri:
        Kii = K[np.ix_(ii, ii)]
        Doi = Dm[ii][:, 1:].T                                # (npo, nri)
        Dog = np.where((gcol < nrt)[None, :], Dm[np.minimum(gcol, nrt - 1)][:, 1:].T, 0.0)
        Kig = K[np.ix_(ii, gcol)]
        Y = np.linalg.solve(Kii, np.hstack([Kig, Doi.T, Fl[ii][:, None]]))
        Yg, YD, YF = Y[:, :ng], Y[:, ng:ng + npo], Y[:, -1]
        Sp = Doi @ YD
        W = Doi @ Yg - Dog
        Z = np.linalg.solve(Sp, np.hstack([W, (Doi @ YF)[:, None]]))
        A = A - Kig.T @ Yg + W.T @ Z[:, :ng]
        Fg = Fg - Kig.T @ YF + W.T @ Z[:, -1]
    d = np.zeros(ng)
    for f in range(3):
        d[f * 2 * nf] = sig[f] * np.sqrt(ln[f])
    A += eps_inv / (0.5 * abs(det)) * np.outer(d, d)
    return A, Fg


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_device_condensation_algebra_matches_oracle(k):
    import paper_2303_06762_gb300 as hdg
    T = hdg.hdg_reference_tables(k)
    m = unit_square(3, shuffle_seed=21)
    t = topo_of(m)
    nu, beta, gamma = 1.3, 0.6, 40.0
    fv = forcing(m, k, curl_bubble_2d(), nu, beta)
    oh = HDG(t, k, nu=nu, beta=beta, gamma=gamma, cache=False)
    for c in range(t.n_cells):
        gv = m.cells[c]
        A, Fc = emulate_cell(m.coords[gv], gv, k, nu, beta, gamma * nu, fv[c], T)
        assert rel(A, oh.element_matrix(c)) < 1e-12, (k, c)
        assert rel(Fc, oh.element_load(c, fv[c])) < 1e-12, (k, c)


def test_reference_tables_basic_identities():
    """R5[i][0]·g_0 = ∫ div phi_i: the facet flux functional (1 for m = 0 moments)."""
    import paper_2303_06762_gb300 as hdg
    for k in range(5):
        T = hdg.hdg_reference_tables(k)
        nf = k + 1
        g0 = np.sqrt(2.0)
        flux = T["R5"][:, 0] / g0
        expect = np.zeros(T["R5"].shape[0])
        for f in range(3):
            expect[f * nf] = 1.0
        assert np.abs(flux - expect).max() < 1e-12


TH = [np.array([-1.0, 1.0]), np.array([0.0, 1.0]), np.array([1.0, 0.0])]   # reference facet edge vectors


def emulate_convection_cell(X, gv, k, nu, eps_inv, T, w, xg_t, bnd, newton):
    npk, nrt, nf = (k + 1) * (k + 2) // 2, (k + 1) * (k + 3), k + 1
    nL, ng, nri, npo = 4 * npk, 6 * nf, k * (k + 1), npk - 1
    ncol = nrt + 3 * nf
    J = np.array([[X[1, 0] - X[0, 0], X[2, 0] - X[0, 0]], [X[1, 1] - X[0, 1], X[2, 1] - X[0, 1]]])
    det = np.linalg.det(J); sgn = 1.0 if det > 0 else -1.0; Ji = np.linalg.inv(J); adet = abs(det)
    ln, nK, tF, sig, o = [], [], [], [], []
    for f, (a, b) in enumerate(FV):
        d = X[b] - X[a]; L = np.hypot(*d); of = 1.0 if gv[a] < gv[b] else -1.0; t = of * d / L
        n = np.array([t[1], -t[0]]); s = 1.0 if n @ (0.5 * (X[a] + X[b]) - X[f]) > 0 else -1.0
        ln.append(L); nK.append(s * n); tF.append(t); sig.append(s); o.append(of)
    sc = np.ones(nrt)
    for f in range(3):
        for m in range(nf):
            sc[f * nf + m] = np.sqrt(ln[f]) * sig[f] * sgn * (o[f] if m % 2 else 1.0)
    C = np.zeros((nL, ncol))
    for c in range(2):
        for e in range(2):
            rows = slice((2 * c + e) * npk, (2 * c + e + 1) * npk)
            vol = sgn * np.einsum("a,b,iabj->ji", J[c], Ji[:, e], T["R1"])
            bd = np.zeros((npk, nrt))
            for f in range(3):
                P = J[c] - nK[f][c] * (nK[f] @ J)
                bd += ln[f] / FL[f] / det * nK[f][e] * np.einsum("a,iaj->ji", P, T["R2"][f])
            C[rows, :nrt] = (vol - bd) * sc[None, :]
            for f in range(3):
                om = np.array([o[f] ** m for m in range(nf)])
                C[rows, nrt + f * nf:nrt + (f + 1) * nf] = nK[f][e] * tF[f][c] * np.sqrt(ln[f]) * T["R3"][f] * om[None, :]
    Dm = sgn * T["R5"] * sc[:, None]
    K = nu / adet * C.T @ C
    JtJ = J.T @ J
    # Picard
    nq = T["R12"].shape[0]; nfq = T["R16"].shape[0]
    uq = T["R11"] @ w
    wh = uq @ Ji.T
    Gq = T["R12"][:, None, None] * np.einsum("qb,qiab->qia", wh, T["R10"])
    Hq = np.einsum("ab,qjb->qja", JtJ, T["R9"])
    Cv = np.zeros((ncol, ncol))
    Cv[:nrt, :nrt] = -np.outer(sc, sc) / adet * np.einsum("qia,qja->ij", Gq, Hq)
    tau = np.zeros((3, nfq, ncol)); aw = np.zeros((3, nfq)); wf = np.zeros((3, nfq, 2))
    for f in range(3):
        for g in range(nfq):
            ph = T["R13"][f, g]                       # (nrt, 2)
            tau[f, g, :nrt] = sc * o[f] / (ln[f] * det) * ((ph @ JtJ.T) @ TH[f])
            for m in range(nf):
                tau[f, g, nrt + f * nf + m] = (o[f] ** m) * T["R15"][g, m] / np.sqrt(ln[f])
            wf[f, g] = T["R14"][f, g] @ w
            aw[f, g] = ln[f] * T["R16"][g] * (wf[f, g] @ nK[f])
    for f in range(3):
        for g in range(nfq):
            a = aw[f, g]; ap, am = max(a, 0.0), min(a, 0.0)
            ti = tau[f, g]
            coef = np.zeros((ncol, ncol))
            coef[:nrt, :nrt] = ap; coef[:nrt, nrt:] = am; coef[nrt:, :nrt] = -ap; coef[nrt:, nrt:] = -am
            Cv += coef * np.outer(ti, ti)
    K += Cv
    Fl = np.zeros(ncol)
    if newton:
        Jtu = uq @ J
        G2 = T["R12"][:, None, None] * np.einsum("qa,qiab->qib", Jtu, T["R10"])
        Cp = np.zeros((ncol, ncol))
        Cp[:nrt, :nrt] = -np.outer(sc, sc) / adet * np.einsum("qib,qjb->ij", G2, T["R9"])
        extra = np.zeros(ncol)
        extra[:nrt] = -sc * sgn * np.einsum("qib,qb->i", G2, wh)
        for f in range(3):
            for g in range(nfq):
                nrm = sc * ((T["R13"][f, g] @ J.T) @ nK[f]) / det
                if (wf[f, g] @ nK[f]) > 1e-10 * np.abs(w).max() and not bnd[f]:
                    wup = wf[f, g] @ tF[f]
                else:
                    wup = xg_t[f] @ tau[f, g, nrt + f * nf:nrt + (f + 1) * nf]
                sr = np.where(np.arange(ncol) < nrt, 1.0, -1.0)
                lw = ln[f] * T["R16"][g]
                Cp[:, :nrt] += lw * np.outer(sr * tau[f, g], nrm) * wup
                extra += sr * aw[f, g] * wup * tau[f, g]
        K += Cp
        Fl += extra
    gcol = []
    for f in range(3):
        gcol += [f * nf + m for m in range(nf)] + [nrt + f * nf + m for m in range(nf)]
    gcol = np.array(gcol); ii = np.arange(3 * nf, nrt)
    A = K[np.ix_(gcol, gcol)].copy(); Fg = Fl[gcol].copy()
    if nri:
        Kii = K[np.ix_(ii, ii)]; Doi = Dm[ii][:, 1:].T
        Dog = np.where((gcol < nrt)[None, :], Dm[np.minimum(gcol, nrt - 1)][:, 1:].T, 0.0)
        Kig = K[np.ix_(ii, gcol)]; Kgi = K[np.ix_(gcol, ii)]
        Y = np.linalg.solve(Kii, np.hstack([Kig, Doi.T, Fl[ii][:, None]]))
        Yg, YD, YF = Y[:, :ng], Y[:, ng:ng + npo], Y[:, -1]
        Sp = Doi @ YD; W = Doi @ Yg - Dog; W2 = Kgi @ YD - Dog.T
        Z = np.linalg.solve(Sp, np.hstack([W, (Doi @ YF)[:, None]]))
        A = A - Kgi @ Yg + W2 @ Z[:, :ng]
        Fg = Fg - Kgi @ YF + W2 @ Z[:, -1]
    d = np.zeros(ng)
    for f in range(3): d[f * 2 * nf] = sig[f] * np.sqrt(ln[f])
    A += eps_inv / (0.5 * adet) * np.outer(d, d)
    return A, Fg


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("newton", [False, True])
def test_device_convection_algebra_matches_oracle(k, newton):
    """The upwind convection (Picard) and Newton blocks as the condensation kernel forms
    them from the point-value tables R9-R16, with LU eliminations, against the oracle."""
    import paper_2303_06762_gb300 as hdg
    from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
    T = hdg.hdg_reference_tables(k)
    m = unit_square(2, shuffle_seed=6)
    t = topo_of(m)
    psi, _ = convecting_stream_2d(1.0)
    w = curl_lattice_2d(m.coords, m.cells, k + 1, psi)
    nu, gamma = 0.05, 50.0
    oh0 = HDG(t, k, nu=nu, gamma=gamma)
    x = np.random.default_rng(3).standard_normal(oh0.n_dof)
    uh = oh0.facet_tangential(x)
    oh = HDG(t, k, nu=nu, gamma=gamma, conv=w, newton_uhat=uh if newton else None)
    for c in range(t.n_cells):
        gv = m.cells[c]
        bnd = [t.interior_index[t.cell_facets[c, f]] < 0 for f in range(3)]
        A, F = emulate_convection_cell(m.coords[gv], gv, k, nu, gamma * nu, T, w[c], uh[c], bnd, newton)
        assert rel(A, oh.element_matrix(c)) < 1e-12, (k, c)
        if newton:
            assert rel(F, oh.element_load(c, np.zeros_like(w[c]))) < 1e-12, (k, c)
