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


def round_sig(x, fmt):
    """Round float64 values to the nearest value of the 16-bit format (ties to even).

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
    return out


def pow2_row_scale(M):
    """Per-row scale s = 2^e with max_j |M_ij| = m 2^e, m in [1/2, 1) (1 for zero rows)."""
    m = np.abs(M).max(axis=1)
    s = np.ones_like(m)
    nz = m > 0
    _, e = np.frexp(m[nz])
    s[nz] = np.ldexp(1.0, e)
    return s


def stored_rows(M, fmt):
    """The value the kernels use for M: each row scaled, rounded, scaled back."""
    s = pow2_row_scale(M)
    return s[:, None] * round_sig(M / s[:, None], fmt)


def rounded_matrix(hdg, fmt):
    """Global matrix assembled from the rounded condensed element matrices."""
    rows, cols, vals = [], [], []
    for c in range(hdg.topo.n_cells):
        idx = hdg.l2g[c]
        m = idx >= 0
        A = stored_rows(hdg.element_matrix(c), fmt)[np.ix_(m, m)]
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
