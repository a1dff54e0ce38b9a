"""Parity of the tensor-core Gram products and block updates (rows a4, a5,
a8, a11) through the C ABI, for both operand formats:

* EIG_ARITH_DF64_TC: double-float blocks, six exact bf16 slices;
* EIG_ARITH_F64_TC: float64 blocks, seven exact bf16 slices, float64 result.

Each product is compared element by element with the exact product (the
definition U^T V, U C, computed to about 2^-64) under the worst-case bound of
tests/tc_bounds.py, and on random data with a statistical check (RMS error
per chunk in units of the chunk maxima) that a product which lost its
lowest kept level would fail.  Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

from oracle import blocks as B
from tc_bounds import exact_matmul, gram_bound, gram_rms_units, update_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_05572_gb300 import _lib as L  # noqa: E402

ARITH = {"df64": L.ARITH_DF64_TC, "f64": L.ARITH_F64_TC}
FMTS = ["df64", "f64"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    yield
    torch.cuda.synchronize()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def to_dev(x, fmt):
    return L.to_df64(dev(x)) if fmt == "df64" else dev(x)


def from_dev(t, fmt):
    return (L.from_df64(t) if fmt == "df64" else t).cpu().numpy()


def tc_gram(U, V, sym, fmt, ldu_pad=0, ldv_pad=0):
    n, a = U.shape
    b = V.shape[1]
    Up = np.zeros((n, a + ldu_pad))
    Up[:, :a] = U
    Ud = to_dev(Up, fmt)
    if V is U and ldv_pad == ldu_pad:
        Vd = Ud
    else:
        Vp = np.zeros((n, b + ldv_pad))
        Vp[:, :b] = V
        Vd = to_dev(Vp, fmt)
    G = torch.full((a, b + 2), 9.0, dtype=torch.float64, device="cuda")
    L.eig_gram(n, a, b, Ud, a + ldu_pad, Vd, b + ldv_pad, ARITH[fmt], sym, G, b + 2)
    assert L.device_status() == 0   # no bounded wait of the product kernel ran out
    assert torch.all(G[:, b:] == 9.0)
    return G[:, :b].cpu().numpy()


def dd_round(X):
    """The double-float image of float64 values (what a DF64 block holds)."""
    hi = X.astype(np.float32).astype(np.float64)
    return hi + (X - hi).astype(np.float32).astype(np.float64)


def operand(X, fmt):
    return dd_round(X) if fmt == "df64" else X


# ---------------------------------------------------------------------------
# Gram G = U^T V
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n,a,b,sym", [(5017, 7, 5, False), (5017, 64, 64, True), (5017, 130, 70, False),
                                       (5017, 150, 150, True), (1, 3, 2, False), (127, 1, 1, True),
                                       (129, 65, 129, False), (3000, 385, 385, True)])
def test_gram_tc_parity(fmt, n, a, b, sym):
    rng = np.random.default_rng(n + a * 7 + b)
    U = rng.standard_normal((n, a))
    V = U if sym else rng.standard_normal((n, b))
    got = tc_gram(U, V, sym, fmt, ldu_pad=3 * (not sym))
    Uo, Vo = operand(U, fmt), operand(V, fmt)
    ref = exact_matmul(Uo.T, Vo)
    err = np.abs(got - ref)
    bound = gram_bound(Uo, Vo, fmt)
    assert np.all(err <= bound), np.max(err / bound)
    if sym:
        assert np.array_equal(got, got.T)


@pytest.mark.parametrize("fmt", FMTS)
def test_gram_tc_statistical_accuracy(fmt):
    """Independent Gaussian columns: the RMS error per chunk is a few
    hundredths of a unit of 2^-53 (float64) or a tenth of 2^-48
    (double-float) times the chunk length and maxima; a product that lost
    its lowest kept level errs by several units (test_slicing_model)."""
    n, a, b = 6000, 96, 80
    rng = np.random.default_rng(77)
    U = rng.standard_normal((n, a))
    V = rng.standard_normal((n, b))
    got = tc_gram(U, V, False, fmt)
    Uo, Vo = operand(U, fmt), operand(V, fmt)
    err = np.abs(got - exact_matmul(Uo.T, Vo))
    rms = gram_rms_units(err, Uo, Vo, fmt)
    print(f"{fmt}: RMS error per chunk {rms:.3f} units")
    assert rms <= 0.5


@pytest.mark.parametrize("fmt", FMTS)
def test_gram_tc_wide_range_and_structure(fmt):
    """Columns scaled by 2^-60 .. 2^60, localized columns (exponential decay
    over thousands of rows, like Anderson eigenvectors), a column with one
    nonzero, a zero column, entries at powers of two with low parts of both
    signs, values just below a power of two, and a sign-alternating column."""
    n, a = 4100, 40
    rng = np.random.default_rng(11)
    U = rng.standard_normal((n, a))
    r = np.arange(n)
    for j in range(8):
        U[:, j] = rng.standard_normal(n) * np.exp(-np.abs(r - 500 * j) / 60.0)
    U[:, 8] = 0.0
    U[:, 9] = 0.0
    U[1234, 9] = -3.75
    U[:, 10] = 2.0 ** rng.integers(-20, 20, n) * (1 + 2.0 ** -30 * rng.choice([-1, 1], n))
    U[:, 11] = np.nextafter(2.0 ** rng.integers(-5, 5, n), 0) * rng.choice([-1.0, 1.0], n)
    U[:, 12] = (-1.0) ** r * (1 + 1e-9 * r)
    for j in range(13, a):
        U[:, j] *= 2.0 ** rng.integers(-60, 60)
    V = rng.standard_normal((n, 24)) * 2.0 ** rng.integers(-30, 30, 24)
    for sym, (X, Y) in ((True, (U, U)), (False, (U, V))):
        got = tc_gram(X, Y, sym, fmt)
        Xo, Yo = operand(X, fmt), operand(Y, fmt)
        err = np.abs(got - exact_matmul(Xo.T, Yo))
        bound = gram_bound(Xo, Yo, fmt)
        assert np.all(err <= bound), np.max(err / np.maximum(bound, 1e-300))
    assert np.all(got[8] == 0.0)


def test_gram_f64_tc_float64_range():
    """Float64 operands beyond the float32 range (2^-900 .. 2^900, columns
    of mixed scale inside one chunk) keep their accuracy; subnormal values
    count as zero."""
    n, a = 1000, 12
    rng = np.random.default_rng(21)
    U = rng.standard_normal((n, a))
    for j in range(a):
        U[:, j] *= 2.0 ** int(rng.integers(-900, 900))
    U[:, 5] = rng.standard_normal(n) * 2.0 ** rng.integers(-400, 400, n)
    V = rng.standard_normal((n, 6)) * 2.0 ** rng.integers(-500, 500, 6)
    got = tc_gram(U, V, False, "f64")
    err = np.abs(got - exact_matmul(U.T, V))
    assert np.all(err <= gram_bound(U, V, "f64")), np.max(err / gram_bound(U, V, "f64"))
    W = np.zeros((n, 2))
    W[:, 0] = 1e-310 * rng.standard_normal(n)    # subnormal: zero chunks
    W[:, 1] = rng.standard_normal(n)
    g = tc_gram(W, W, True, "f64")
    assert np.all(g[0] == 0.0) and np.all(g[:, 0] == 0.0)
    assert abs(g[1, 1] - np.dot(W[:, 1], W[:, 1])) <= 1e-14 * np.dot(W[:, 1], W[:, 1])


def test_gram_f64_tc_nan_propagates():
    n, a = 700, 5
    U = np.random.default_rng(3).standard_normal((n, a))
    U[345, 2] = np.nan
    g = tc_gram(U, U, True, "f64")
    assert np.all(np.isnan(g[2])) and np.all(np.isnan(g[:, 2]))
    assert np.all(np.isfinite(np.delete(np.delete(g, 2, 0), 2, 1)))


def test_gram_df64_tc_tiny_chunks_are_zero_and_deterministic():
    n, a = 3000, 20
    rng = np.random.default_rng(5)
    U = rng.standard_normal((n, a))
    U[:, 3] = 1e-35 * rng.standard_normal(n)   # every chunk maximum below 2^-100
    g1 = tc_gram(U, U, True, "df64")
    g2 = tc_gram(U, U, True, "df64")
    assert np.array_equal(g1, g2)
    assert np.all(g1[3] == 0.0) and np.all(g1[:, 3] == 0.0)


@pytest.mark.parametrize("fmt", FMTS)
def test_gram_tc_deterministic(fmt):
    n, a, b = 9000, 100, 70
    rng = np.random.default_rng(8)
    U = rng.standard_normal((n, a))
    V = rng.standard_normal((n, b))
    assert np.array_equal(tc_gram(U, V, False, fmt), tc_gram(U, V, False, fmt))


@pytest.mark.parametrize("fmt", FMTS)
def test_gram_tc_orthonormal_columns(fmt):
    """The CholeskyQR Gram of an orthonormal block: within 1e-13 of the
    identity's exact Gram (float64: 4e-15), like the CUDA-core products."""
    n, a = 20000, 96
    Q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((n, a)))
    Qd = to_dev(Q, fmt)
    G = torch.empty(a, a, dtype=torch.float64, device="cuda")
    L.eig_gram(n, a, a, Qd, a, Qd, a, ARITH[fmt], True, G, a)
    Qo = operand(Q, fmt)
    ref = exact_matmul(Qo.T, Qo)
    assert np.max(np.abs(G.cpu().numpy() - ref)) <= (1e-13 if fmt == "df64" else 4e-15)


# ---------------------------------------------------------------------------
# Update Y = U C + beta Y
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n,s,c,beta", [(5017, 7, 5, 0.0), (5017, 64, 64, 1.0), (5017, 130, 70, -0.37),
                                        (3001, 385, 257, 0.0), (1, 3, 2, 2.5), (65, 1, 129, -1.0),
                                        (4099, 1201, 33, 0.5)])
def test_update_tc_parity(fmt, n, s, c, beta):
    rng = np.random.default_rng(n + s * 3 + c)
    U = rng.standard_normal((n, s)) * 2.0 ** rng.integers(-20, 20, s)
    Cm = rng.standard_normal((s, c))
    Y0 = rng.standard_normal((n, c))
    Yd = to_dev(Y0, fmt)
    L.eig_block_update(n, s, c, to_dev(U, fmt), s, dev(Cm), c, Yd, c, beta, ARITH[fmt])
    assert L.device_status() == 0
    got = from_dev(Yd, fmt)
    Uo, Yo = operand(U, fmt), operand(Y0, fmt)
    ref = exact_matmul(Uo, Cm) + beta * Yo
    bound = update_bound(Uo, Cm, beta, Yo, fmt)
    err = np.abs(got - ref)
    assert np.all(err <= bound), np.max(err / bound)


@pytest.mark.parametrize("fmt", FMTS)
def test_update_tc_zero_width_and_padding(fmt):
    """s = 0 gives beta Y; the leading dimensions larger than the widths are
    neither read nor written."""
    n, s, c = 300, 40, 20
    rng = np.random.default_rng(4)
    U = np.zeros((n, s + 5))
    U[:, :s] = rng.standard_normal((n, s))
    U[:, s:] = np.nan
    Cm = np.zeros((s, c + 3))
    Cm[:, :c] = rng.standard_normal((s, c))
    Cm[:, c:] = np.nan
    Y0 = rng.standard_normal((n, c + 2))
    Yd = to_dev(Y0, fmt)
    L.eig_block_update(n, s, c, to_dev(U, fmt), s + 5, dev(Cm), c + 3, Yd, c + 2, 0.5, ARITH[fmt])
    got = from_dev(Yd, fmt)
    Uo, Yo = operand(U[:, :s], fmt), operand(Y0, fmt)
    ref = Uo @ Cm[:, :c] + 0.5 * Yo[:, :c]
    assert np.all(np.abs(got[:, :c] - ref) <= 1e-12 * (np.abs(Uo) @ np.abs(Cm[:, :c]) + np.abs(Yo[:, :c])))
    assert np.array_equal(got[:, c:], Yo[:, c:])
    Yd = to_dev(Y0, fmt)
    L.eig_block_update(n, 0, c, to_dev(U, fmt), s + 5, dev(Cm), c + 3, Yd, c + 2, -2.0, ARITH[fmt])
    assert np.allclose(from_dev(Yd, fmt)[:, :c], -2.0 * Yo[:, :c], rtol=1e-14)


def test_update_f64_tc_segmented_output_matches_plain():
    """The solver writes X and P of one update into two column segments of S
    (ld = 3 k_max); through the C ABI the same product on a strided output
    with ld > c gives the same values as on a packed one."""
    n, s, c = 2000, 200, 96
    rng = np.random.default_rng(12)
    U = rng.standard_normal((n, s))
    Cm = rng.standard_normal((s, c))
    Y1 = torch.zeros(n, c, dtype=torch.float64, device="cuda")
    Y2 = torch.zeros(n, 3 * c + 4, dtype=torch.float64, device="cuda")
    Ud = dev(U)
    L.eig_block_update(n, s, c, Ud, s, dev(Cm), c, Y1, c, 0.0, L.ARITH_F64_TC)
    L.eig_block_update(n, s, c, Ud, s, dev(Cm), c, Y2[:, c + 4:], 3 * c + 4, 0.0, L.ARITH_F64_TC)
    assert torch.equal(Y1, Y2[:, c + 4:2 * c + 4])
    assert torch.count_nonzero(Y2[:, :c + 4]) == 0 and torch.count_nonzero(Y2[:, 2 * c + 4:]) == 0


# ---------------------------------------------------------------------------
# bounded waits
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", FMTS)
def test_bounded_wait_runs_out_and_the_next_call_is_clean(fmt):
    """The self-test entry point withholds one pipeline stage of a product,
    so the MMA issuer's bounded wait runs out (no fault, no hang); the
    device status reports it once, and the next product is exact again."""
    assert L.device_status() == 0
    L.eig_tc_wait_selftest(ARITH[fmt], 0.05)
    assert L.device_status() == L.EIG_ETIMEOUT
    assert L.device_status() == 0
    n, a = 3000, 70
    U = np.random.default_rng(6).standard_normal((n, a))
    got = tc_gram(U, U, True, fmt)
    Uo = operand(U, fmt)
    assert np.all(np.abs(got - exact_matmul(Uo.T, Uo)) <= gram_bound(Uo, Uo, fmt))
