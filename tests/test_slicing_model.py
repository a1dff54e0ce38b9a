"""The error model of the tensor-core products of double-float blocks, checked
on the CPU from the definition of the splitting (Ozaki, Ogita, Oishi and
Rump, Numer. Algorithms 59, 2012, in its fixed-point form), independently of
the GPU kernels.  The GPU parity tests allow 32 * 2^-48 of the chunk maxima
per contraction index (tests/tc_bounds.py); this module shows why that bound
holds:

* a value v = hi + lo (two float32) scaled by 2^(7 - e), with 2^(e-1) <= the
  chunk's max |hi| < 2^e, is cut by six round-to-nearest steps (each in
  float32 with an error-free TwoSum of the remainder, times 256) into
  integers |s_q| <= 128, and the six slices represent v to 2^-41 of the
  scaled value;
* the product of two chunks keeps the slice pairs with q_a + q_b <= 5; each
  level sum is an integer below 2^24 (exact in an fp32 accumulator); the
  kept levels differ from the exact dot product by at most about
  28 * 2^-48 * (chunk length) * max|a| max|b|.
Everything here is exact rational arithmetic (Python integers / fractions)
except the float32 steps of the cut, which numpy performs with IEEE rounding.
"""
from fractions import Fraction

import numpy as np
import pytest

CH = 128
S = 6


def two_sum32(a, b):
    s = np.float32(a + b)
    z = np.float32(s - a)
    e = np.float32(np.float32(a - np.float32(s - z)) + np.float32(b - z))
    return s, e


def chunk_exp(hi):
    m = float(np.max(np.abs(hi)))
    if m < 2.0 ** -100:
        return None
    _, e = np.frexp(m)          # 2^(e-1) <= m < 2^e
    return int(e)


def cut(h, l, e):
    """Six slices of the double-float value (h, l) against exponent e."""
    sc = np.float32(2.0 ** (7 - e))
    h = np.float32(h * sc)
    l = np.float32(l * sc)
    out = []
    for _ in range(S):
        r = np.float32(np.rint(h))
        out.append(int(r))
        nh, nl = two_sum32(np.float32(h - r), l)
        h = np.float32(nh * np.float32(256.0))
        l = np.float32(nl * np.float32(256.0))
    return out


def dd_values(rng, n, spread):
    """n double-float values (hi, lo) with magnitudes spread over 2^+-spread."""
    x = rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def exact(h, l):
    return Fraction(float(h)) + Fraction(float(l))


@pytest.mark.parametrize("spread", [0, 4, 20])
def test_slices_are_bf16_integers_and_represent_the_value(spread):
    rng = np.random.default_rng(spread)
    hi, lo = dd_values(rng, CH, spread)
    e = chunk_exp(hi)
    for h, l in zip(hi, lo):
        s = cut(h, l, e)
        assert all(abs(q) <= 128 for q in s)       # 8 bits: exact in bf16
        rep = sum(Fraction(q, 256 ** i) for i, q in enumerate(s))
        scaled = exact(h, l) * Fraction(2) ** (7 - e)
        assert abs(rep - scaled) <= Fraction(1, 2 ** 41)


def level_sums(sa, sb):
    """Exact integer level sums L_l = sum_k sum_{i+j=l} sa[k][i] sb[k][j]."""
    L = [0] * S
    for a, b in zip(sa, sb):
        for i in range(S):
            for j in range(S - i):
                L[i + j] += a[i] * b[j]
    return L


@pytest.mark.parametrize("seed,spread", [(0, 0), (1, 3), (2, 12), (3, 0)])
def test_kept_levels_bound_the_chunk_product(seed, spread):
    rng = np.random.default_rng(seed)
    ha, la = dd_values(rng, CH, spread)
    hb, lb = dd_values(rng, CH, spread)
    if seed == 3:   # adversarial: every value just below the chunk maximum
        ha = np.full(CH, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))))
        hb = ha.copy()
        la = np.full(CH, np.float32(2.0 ** -25))
        lb = la.copy()
    ea, eb = chunk_exp(ha), chunk_exp(hb)
    sa = [cut(h, l, ea) for h, l in zip(ha, la)]
    sb = [cut(h, l, eb) for h, l in zip(hb, lb)]
    L = level_sums(sa, sb)
    for l in range(S):
        assert abs(L[l]) < 2 ** 24                 # exact in fp32, any order
        assert abs(L[l]) <= (l + 1) * CH * 2 ** 14
    kept = sum(Fraction(L[l], 256 ** l) for l in range(S)) * Fraction(2) ** (ea - 7 + eb - 7)
    dot = sum(exact(a, b) * exact(c, d) for a, b, c, d in zip(ha, la, hb, lb))
    Ma = max(abs(exact(a, b)) for a, b in zip(ha, la))
    Mb = max(abs(exact(c, d)) for c, d in zip(hb, lb))
    err = abs(kept - dot)
    assert err <= Fraction(28, 2 ** 48) * CH * Ma * Mb


def chunk_errors(seed, levels):
    """|kept - exact| of one random chunk product in units of
    2^-48 * CH * max|a| max|b|, keeping the levels < `levels`."""
    rng = np.random.default_rng(seed)
    ha, la = dd_values(rng, CH, 0)
    hb, lb = dd_values(rng, CH, 0)
    ea, eb = chunk_exp(ha), chunk_exp(hb)
    L = level_sums([cut(h, l, ea) for h, l in zip(ha, la)], [cut(h, l, eb) for h, l in zip(hb, lb)])
    kept = sum(Fraction(L[l], 256 ** l) for l in range(levels)) * Fraction(2) ** (ea - 7 + eb - 7)
    dot = sum(exact(a, b) * exact(c, d) for a, b, c, d in zip(ha, la, hb, lb))
    Ma = max(abs(exact(a, b)) for a, b in zip(ha, la))
    Mb = max(abs(exact(c, d)) for c, d in zip(hb, lb))
    return float(abs(kept - dot) / (Fraction(1, 2 ** 48) * CH * Ma * Mb))


def test_typical_error_is_far_below_the_bound_and_a_lost_level_is_not():
    """On random chunks the six kept levels err by about 0.1 unit (RMS), two
    orders below the worst-case 28; a product that lost its top level
    (level 5, a planted mistake of this model) errs by about 20 units, which
    the worst-case bound alone would not reveal."""
    full = np.array([chunk_errors(s, S) for s in range(100, 116)])
    lost = np.array([chunk_errors(s, S - 1) for s in range(100, 116)])
    assert np.sqrt(np.mean(full ** 2)) <= 1.0
    assert np.sqrt(np.mean(lost ** 2)) >= 4.0
