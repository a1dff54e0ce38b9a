"""The exact-product reference of the tensor-core parity tests
(tc_bounds.exact_matmul) against rational arithmetic: on small matrices
with entries spread over 2^-300 .. 2^300, zero rows and columns, cancelling
sums and a localized column, its error stays inside its stated allowance
(2^-70 of the 64-index chunk maxima per index), and where the entries of a
chunk are of one scale, inside 2^-66 of |A| @ |B|."""
from fractions import Fraction

import numpy as np
import pytest

from tc_bounds import exact_matmul, ref_allowance


def exact_fraction(A, B):
    m, k = A.shape
    n = B.shape[1]
    out = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            out[i, j] = float(sum(Fraction(float(A[i, t])) * Fraction(float(B[t, j])) for t in range(k)))
    return out


@pytest.mark.parametrize("seed,spread", [(0, 0), (1, 30), (2, 300)])
def test_exact_matmul_matches_rational_arithmetic(seed, spread):
    rng = np.random.default_rng(seed)
    m, k, n = 5, 150, 4
    A = rng.standard_normal((m, k)) * 2.0 ** rng.integers(-spread, spread + 1, (m, k))
    B = rng.standard_normal((k, n)) * 2.0 ** rng.integers(-spread, spread + 1, (k, n))
    A[1] = 0.0
    B[:, 2] = -A[0] * 2.0 ** -3          # row 0 times column 2 cancels to a small sum
    A[0, 77] += 1e-10
    B[:, 3] = np.exp(-np.abs(np.arange(k) - 40) / 3.0)   # localized column
    ref = exact_fraction(A, B)
    got = exact_matmul(A, B)
    err = np.abs(got - ref)
    assert np.all(err <= ref_allowance(A, B))
    if spread == 0:
        assert np.all(err <= 2.0 ** -66 * (np.abs(A) @ np.abs(B)))
    assert np.all(got[1] == 0.0)
