"""Error bounds of the tensor-core products, shared by the GPU parity tests.

Every value is cut into 8-bit slices against a power-of-two scale shared by
a 128-index chunk of the contraction; the slice pairs of the kept levels are
summed exactly and the rest dropped (tests/test_slicing_model.py derives the
constants on the CPU from the definition of the splitting).

* double-float blocks (EIG_ARITH_DF64_TC, six slices, levels 0..5): per
  contraction index at most about 28 * 2^-48 of the product of the two chunk
  maxima, plus the double-float accumulation (1e-12 relative to
  sum |u v|).  The tests allow 32 * 2^-48.
* float64 blocks (EIG_ARITH_F64_TC, seven slices, levels 0..6): per chunk at
  most 8 units of 2^-53 * (chunk length) * max|u| max|v|, the triple-float
  accumulation below 2^-53 of sum |c_k|, then float64 roundings: the final
  conversion and the fixed-order sum of at most `nsplit` split-K partials.
  The tests allow 10 units per chunk and (nsplit + 4) * 2^-53 relative to
  sum |u v|.

The reference is the exact product to about 2^-70 (exact_matmul, an exact
digit splitting evaluated with float64 BLAS and a double-double sum; pinned
against rational arithmetic in tests/test_tc_reference.py).
"""
import numpy as np

CHUNK = 128
SLICE_TOL = {"df64": 32 * 2.0 ** -48, "f64": 10 * 2.0 ** -53}
DF64_RTOL = 1e-12
U53 = 2.0 ** -53


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


def _two_sum(a, b):
    s = a + b
    z = s - a
    return s, (a - (s - z)) + (b - z)


def exact_matmul(A, B, chunk=64, nsl=4, bits=18):
    """A @ B to about 2^-70 of the chunk maxima (ref_allowance) in float64
    arithmetic: per chunk of
    64 contraction indices every row of A and column of B is scaled by a
    power of two below its maximum and cut into four 18-bit integer digits;
    each digit product is a sum of 64 integer products below 2^36, exact in
    float64 whatever order BLAS adds in; the digit products are scaled back
    and summed in double-double (TwoSum)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, K = A.shape
    n = B.shape[1]
    hi = np.zeros((m, n))
    lo = np.zeros((m, n))

    def digits(X, axis):
        mx = np.max(np.abs(X), axis=axis, keepdims=True)
        _, e = np.frexp(np.where(mx > 0, mx, 1.0))      # max < 2^e
        t = np.ldexp(X, -e)                             # |t| < 1, exact
        out = []
        for _ in range(nsl):
            t = np.ldexp(t, bits)
            d = np.rint(t)
            out.append(d)
            t = t - d                                   # exact remainder
        return out, e

    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        for c0 in range(0, K, chunk):
            Da, ea = digits(A[:, c0:c0 + chunk], 1)
            Db, eb = digits(B[c0:c0 + chunk, :], 0)
            esum = ea + eb                              # (m, 1) + (1, n)
            for i in range(nsl):
                for j in range(nsl):
                    P = Da[i] @ Db[j]                   # exact integers
                    x = np.ldexp(P, esum - bits * (i + j + 2))
                    hi, e1 = _two_sum(hi, x)
                    lo = lo + e1
    return hi + lo


def ref_allowance(A, B, chunk=64):
    """Error allowance of exact_matmul itself: four 18-bit digits leave
    2^-73 of the chunk maximum per value, so per contraction index at most
    2^-71 of the product of the two 64-index chunk maxima, plus the
    double-double sum."""
    K = A.shape[1]
    tot = np.zeros((A.shape[0], B.shape[1]))
    for c0 in range(0, K, chunk):
        ma = np.max(np.abs(A[:, c0:c0 + chunk]), axis=1, keepdims=True)
        mb = np.max(np.abs(B[c0:c0 + chunk, :]), axis=0, keepdims=True)
        tot += min(chunk, K - c0) * (ma * mb)
    return 2.0 ** -70 * tot + 2.0 ** -100 * (np.abs(A) @ np.abs(B))


def nsplit_max(n):
    return min(152, -(-n // CHUNK))


def gram_bound(U, V, fmt="df64"):
    """Allowed |G - U^T V| entrywise for the tensor-core Gram (chunks run
    over the rows)."""
    Mu, cnt = chunk_max(U)
    Mv, _ = chunk_max(V)
    slicing = SLICE_TOL[fmt] * ((Mu * cnt[:, None]).T @ Mv)
    absuv = np.abs(U).T @ np.abs(V)
    if fmt == "df64":
        return DF64_RTOL * absuv + slicing + ref_allowance(U.T, V)
    return (nsplit_max(U.shape[0]) + 4) * U53 * absuv + slicing + ref_allowance(U.T, V)


def update_bound(U, Cm, beta=0.0, Y0=None, fmt="df64"):
    """Allowed |Y - (U C + beta Y0)| entrywise for the tensor-core update
    (chunks run over the columns of U and the rows of C)."""
    Mu, cnt = row_chunk_max(U)
    Mc, _ = row_chunk_max(Cm.T)
    slicing = SLICE_TOL[fmt] * ((Mu * cnt) @ Mc.T)
    absuc = np.abs(U) @ np.abs(Cm)
    rt = DF64_RTOL if fmt == "df64" else 4 * U53
    b = rt * absuc + slicing + ref_allowance(U, Cm)
    if beta != 0.0:
        b = b + rt * abs(beta) * np.abs(Y0)
    return b


def gram_rms_units(err, U, V, fmt):
    """RMS over the entries of err / (unit * sqrt(sum over chunks of
    (count * M_u * M_v)^2)): the chunk errors add like a random walk, so on
    random data this is the typical error per chunk in units of
    unit * (chunk length) * M_u M_v (unit 2^-48 for double-float, 2^-53 for
    float64)."""
    Mu, cnt = chunk_max(U)
    Mv, _ = chunk_max(V)
    unit = 2.0 ** -48 if fmt == "df64" else U53
    den = unit * np.sqrt(((Mu * cnt[:, None]) ** 2).T @ (Mv ** 2))
    return float(np.sqrt(np.mean((err / den) ** 2)))
