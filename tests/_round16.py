"""CPU model of the 16-bit matrix copies of the HDG_MIXED_BF16 / HDG_MIXED_FP16
preconditioners, for the parity tests (test infrastructure).

The library stores every row of the order-k condensed element matrices and of
the patch inverses as s · Â with s a power of two (the row's largest entry
m·2^e, m in [1/2, 1), gives s = 2^e) and Â rounded to nearest-even in the
16-bit format.  This module rounds FP64 values the same way from their binary
expansion (no library conversion), and builds an oracle hp-multigrid whose
order-k smoother and residual read such rounded matrices.
"""
import numpy as np
import scipy.sparse as sp

# significant bits and smallest normal exponent of each format
FORMATS = {"fp16": (11, -14), "bf16": (8, -126)}


def round_sig(x, fmt, ftz=False):
    """Round float64 values to the nearest value of the 16-bit format (ties to even);
    with ftz, results below the smallest normal value become zero.

    Values must lie below the format's largest finite value (|x| < 1 here).
    """
    bits, emin = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    _, e = np.frexp(np.abs(x[nz]))                  # |x| = m 2^e, m in [1/2, 1)
    e = np.maximum(e - 1, emin)                     # exponent of the leading bit, subnormals clamp
    ulp = np.ldexp(1.0, e - (bits - 1))
    out[nz] = np.round(x[nz] / ulp) * ulp           # x / ulp is exact; np.round ties to even
    if ftz:
        out[np.abs(out) < np.ldexp(1.0, emin)] = 0.0
    return out


def pow2_row_scale(M):
    """Per-row scale s = 2^e with max_j |M_ij| = m 2^e, m in [1/2, 1) (1 for zero rows)."""
    m = np.abs(M).max(axis=1)
    s = np.ones_like(m)
    nz = m > 0
    _, e = np.frexp(m[nz])
    s[nz] = np.ldexp(1.0, e)
    return s


def stored_rows(M, fmt, ftz=False):
    """The value the kernels use for M: each row scaled, rounded, scaled back."""
    s = pow2_row_scale(M)
    return s[:, None] * round_sig(M / s[:, None], fmt, ftz)


def rounded_matrix(hdg, fmt, ftz=False):
    """Global matrix assembled from the rounded condensed element matrices."""
    rows, cols, vals = [], [], []
    for c in range(hdg.topo.n_cells):
        idx = hdg.l2g[c]
        m = idx >= 0
        A = stored_rows(hdg.element_matrix(c), fmt, ftz)[np.ix_(m, m)]
        I = idx[m]
        rows.append(np.repeat(I, len(I)))
        cols.append(np.tile(I, len(I)))
        vals.append(A.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(hdg.n_dof, hdg.n_dof))


def round_hpmg(M, fmt):
    """Make the order-k part of an oracle MG_hp read the rounded copies (in place)."""
    Ar = rounded_matrix(M.hdg, fmt)
    M.A = Ar
    M.gs.A = Ar
    M.gs.rows = [Ar[d, :] for _, d in M.gs.patches]
    M.gs.inv = [stored_rows(Ai, fmt) for Ai in M.gs.inv]
    return M


def _col_round(v, fmt, ftz=False):
    """Round a column to the 16-bit format after a power-of-two scale that brings its
    largest magnitude into [1/2, 1) (the batched kernels' per-column scaling)."""
    s = pow2_row_scale(np.asarray(v, dtype=np.float64)[None, :])[0]
    return s * round_sig(v / s, fmt, ftz)


def round_hpmg_tc(M, fmt, ftz=False):
    """Make the order-k smoother of an oracle MG_hp follow the batched tensor-core
    sweep for one column (in place): rounded element rows and inverses as in
    round_hpmg, the star's gathered unknowns and the patch residual each rounded
    per column; the residual before Π_k^0 stays exact (FP32 on the device)."""
    hdg = M.hdg
    topo = hdg.topo
    Ar = rounded_matrix(hdg, fmt, ftz)
    gs = M.gs
    inv = [stored_rows(Ai, fmt, ftz) for Ai in gs.inv]
    rows = [Ar[d, :] for _, d in gs.patches]
    cells_of = [[] for _ in range(topo.coords.shape[0])]
    for c, cv in enumerate(topo.cells):
        for v in cv:
            cells_of[v].append(c)
    stars = []
    for v, _ in gs.patches:
        idx = np.concatenate([hdg.l2g[c] for c in cells_of[v]])
        stars.append(np.unique(idx[idx >= 0]))

    def step(g, u, i):
        d = gs.patches[i][1]
        xq = u.copy()
        xq[stars[i]] = _col_round(u[stars[i]], fmt, ftz)
        r = g[d] - rows[i] @ xq
        u[d] += inv[i] @ _col_round(r, fmt, ftz)

    def forward(g, u):
        for i in range(len(gs.patches)):
            step(g, u, i)
        return u

    def backward(g, u):
        for i in reversed(range(len(gs.patches))):
            step(g, u, i)
        return u

    gs.forward, gs.backward = forward, backward
    return M
