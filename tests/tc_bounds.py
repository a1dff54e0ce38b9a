"""Error bounds of the tensor-core products of double-float blocks
(EIG_ARITH_DF64_TC), shared by the GPU parity tests.

Every value is cut into six 8-bit slices against a power-of-two scale shared
by a 128-index chunk of the contraction; the slice pairs of levels 0..5 are
summed exactly and the rest dropped.  Per contraction index the error is at
most about 28 * 2^-48 of the product of the two chunk maxima (20 from the
dropped levels, 8 from the six-slice representation), plus the double-float
accumulation (1e-12 relative to sum |u v|).  The tests allow 32 * 2^-48.
"""
import numpy as np

CHUNK = 128
SLICE_TOL = 32 * 2.0 ** -48
DF64_RTOL = 1e-12


def chunk_max(X, rows=CHUNK):
    """max |x| over each column's chunks of `rows` rows: (chunks, cols), and
    the number of rows in each chunk (the last one ragged)."""
    n = X.shape[0]
    nch = -(-n // rows)
    P = np.zeros((nch * rows, X.shape[1]))
    P[:n] = np.abs(X)
    cnt = np.full(nch, rows, dtype=np.float64)
    cnt[-1] = n - (nch - 1) * rows
    return P.reshape(nch, rows, -1).max(axis=1), cnt


def row_chunk_max(X, cols=CHUNK):
    """max |x| over each row's chunks of `cols` columns: (rows, chunks), and
    the number of columns in each chunk."""
    m, k = X.shape
    nch = -(-k // cols)
    P = np.zeros((m, nch * cols))
    P[:, :k] = np.abs(X)
    cnt = np.full(nch, cols, dtype=np.float64)
    cnt[-1] = k - (nch - 1) * cols
    return P.reshape(m, nch, cols).max(axis=2), cnt


def gram_bound(U, V):
    """Allowed |G - U^T V| entrywise for the tensor-core Gram (chunks run
    over the rows)."""
    Mu, cnt = chunk_max(U)
    Mv, _ = chunk_max(V)
    return DF64_RTOL * (np.abs(U).T @ np.abs(V)) + SLICE_TOL * ((Mu * cnt[:, None]).T @ Mv)


def update_bound(U, Cm, beta=0.0, Y0=None):
    """Allowed |Y - (U C + beta Y0)| entrywise for the tensor-core update
    (chunks run over the columns of U and the rows of C)."""
    Mu, cnt = row_chunk_max(U)
    Mc, _ = row_chunk_max(Cm.T)
    b = DF64_RTOL * (np.abs(U) @ np.abs(Cm)) + SLICE_TOL * ((Mu * cnt) @ Mc.T)
    if beta != 0.0:
        b = b + DF64_RTOL * abs(beta) * np.abs(Y0)
    return b
