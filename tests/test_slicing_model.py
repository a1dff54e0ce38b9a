"""The error model of the tensor-core products of double-float and float64
blocks, checked on the CPU from the definition of the splitting (Ozaki,
Ogita, Oishi and Rump, Numer. Algorithms 59, 2012, in its fixed-point form),
independently of the GPU kernels.  The GPU parity tests use the bounds of
tests/tc_bounds.py; this module shows why they hold.

Double-float blocks (six slices):

* a value v = hi + lo (two float32) scaled by 2^(7 - e), with 2^(e-1) <= the
  chunk's max |hi| < 2^e, is cut by six round-to-nearest steps (each in
  float32 with an error-free TwoSum of the remainder, times 256) into
  integers |s_q| <= 128, and the six slices represent v to 2^-41 of the
  scaled value;
* the product of two chunks keeps the slice pairs with q_a + q_b <= 5; each
  level sum is an integer below 2^24 (exact in an fp32 accumulator); the
  kept levels differ from the exact dot product by at most about
  28 * 2^-48 * (chunk length) * max|a| max|b|.

Float64 blocks (seven slices, second half of this module):

* F = x 2^(55 - e) as an integer from the bit pattern, balanced base-256
  digits |d_q| <= 128, the value represented to 2^-49 of the scaled value;
* levels 0..6 kept (28 slice pairs), level sums below 2^24; the float32
  combination gives hi + lo exactly equal to levels 0..3; the chunk value
  errs by at most 8 units of 2^-53 * (chunk length) * max|a| max|b|;
* the triple-float accumulation of chunk values is float64-class.

Everything here is exact rational arithmetic (Python integers / fractions)
except the float32 steps, which numpy performs with IEEE rounding.
"""
import math
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


# ---------------------------------------------------------------------------
# Float64 blocks: seven slices cut from the bit pattern, levels 0..6 kept,
# the seven level sums combined in float32 into hi + lo (exact) + small, and
# the chunk values accumulated in triple-float.
# ---------------------------------------------------------------------------
S7 = 7


def f64_parts(x):
    """(sign, biased exponent, 53-bit integer mantissa) of a normal float64."""
    b = int(np.float64(x).view(np.uint64))
    return b >> 63, (b >> 52) & 0x7FF, (b & ((1 << 52) - 1)) | (1 << 52)


def chunk_emax(xs):
    """Largest biased exponent of the chunk (0: all zero)."""
    return max((f64_parts(x)[1] for x in xs if x != 0.0), default=0)


def cut7(x, emax):
    """Seven balanced base-256 digits of F = x 2^(55 - e), e = emax - 1022,
    right shifts rounded half away from zero (the definition, in integers)."""
    if x == 0.0 or emax == 0:
        return [0] * S7
    sgn, E, m = f64_parts(x)
    sh = E - emax + 2
    u = m << sh if sh >= 0 else ((m + (1 << (-sh - 1))) >> (-sh) if sh > -60 else 0)
    F = -u if sgn else u
    d = []
    for _ in range(S7 - 1):
        q = ((F + 128) & 255) - 128
        d.append(q)
        F = (F - q) >> 8
    d.append(F)
    return d[::-1]            # d[0] most significant


def f64_values(rng, n, spread):
    return rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)


@pytest.mark.parametrize("spread", [0, 6, 40])
def test_f64_slices_are_bf16_integers_and_represent_the_value(spread):
    rng = np.random.default_rng(10 + spread)
    x = f64_values(rng, CH, spread)
    emax = chunk_emax(x)
    e = emax - 1022
    assert 2.0 ** (e - 1) <= np.max(np.abs(x)) < 2.0 ** e
    for v in x:
        d = cut7(v, emax)
        assert all(abs(q) <= 128 for q in d)
        rep = sum(Fraction(q, 256 ** i) for i, q in enumerate(d))
        assert abs(rep - Fraction(float(v)) * Fraction(2) ** (7 - e)) <= Fraction(1, 2 ** 49)


def level_sums7(da, db):
    L = [0] * S7
    for a, b in zip(da, db):
        for i in range(S7):
            for j in range(S7 - i):
                L[i + j] += a[i] * b[j]
    return L


def combine7_f32(L):
    """The flush's combination of the prescaled level sums a_l = L_l 2^-8l
    in float32: magic-constant split of levels 1..3 at multiples of 1/2."""
    a = [np.float32(Fraction(L[l], 256 ** l)) for l in range(S7)]
    for l in range(S7):    # prescaled level sums are exact in float32
        assert Fraction(float(a[l])) == Fraction(L[l], 256 ** l)
    MAGIC = np.float32(1.5 * 2 ** 22)
    h = [np.float32(np.float32(a[l] + MAGIC) - MAGIC) for l in (1, 2, 3)]
    hi = np.float32(np.float32(a[0] + h[0]) + np.float32(h[1] + h[2]))
    lo = np.float32(np.float32(np.float32(a[1] - h[0]) + np.float32(a[2] - h[1])) + np.float32(a[3] - h[2]))
    small = np.float32(np.float32(a[4] + a[5]) + a[6])
    return hi, lo, small


def f64_chunk(rng, spread, adversarial=False):
    xa = f64_values(rng, CH, spread)
    xb = f64_values(rng, CH, spread)
    if adversarial:   # every value at the largest digits of the chunk
        xa = np.full(CH, np.nextafter(1.0, 0.0))
        xb = -xa
    ea, eb = chunk_emax(xa), chunk_emax(xb)
    L = level_sums7([cut7(v, ea) for v in xa], [cut7(v, eb) for v in xb])
    scale = Fraction(2) ** ((ea - 1022) - 7 + (eb - 1022) - 7)
    dot = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(xa, xb))
    unit = Fraction(1, 2 ** 53) * CH * Fraction(float(np.max(np.abs(xa)))) * Fraction(float(np.max(np.abs(xb))))
    return L, scale, dot, unit


@pytest.mark.parametrize("seed,spread,adv", [(20, 0, False), (21, 3, False), (22, 30, False), (23, 0, True)])
def test_f64_kept_levels_and_combination_bound_the_chunk_product(seed, spread, adv):
    """Level sums are integers below 2^24; hi + lo reproduces levels 0..3
    exactly; the value hi + lo + small differs from the exact dot product by
    at most 8 units of 2^-53 * CH * max|a| max|b|."""
    L, scale, dot, unit = f64_chunk(np.random.default_rng(seed), spread, adv)
    for l in range(S7):
        assert abs(L[l]) <= (l + 1) * CH * 2 ** 14 < 2 ** 24
    hi, lo, small = combine7_f32(L)
    assert Fraction(float(hi)) + Fraction(float(lo)) == sum(Fraction(L[l], 256 ** l) for l in range(4))
    got = (Fraction(float(hi)) + Fraction(float(lo)) + Fraction(float(small))) * scale
    assert abs(got - dot) <= 8 * unit


def f64_chunk_error(seed, levels):
    L, scale, dot, unit = f64_chunk(np.random.default_rng(seed), 0)
    kept = sum(Fraction(L[l], 256 ** l) for l in range(levels)) * scale
    return float(abs(kept - dot) / unit)


def test_f64_typical_error_and_a_lost_level():
    """Random chunks: about 0.02 unit of 2^-53 CH max|a| max|b| (RMS); a
    product that dropped level 6 (a planted mistake of this model) errs by
    about 4.5 units, so an RMS check at 0.25 units separates the two."""
    full = np.array([f64_chunk_error(s, S7) for s in range(200, 212)])
    lost = np.array([f64_chunk_error(s, S7 - 1) for s in range(200, 212)])
    assert np.sqrt(np.mean(full ** 2)) <= 0.25
    assert np.sqrt(np.mean(lost ** 2)) >= 2.0


def two_sum_f32(a, b):
    s = np.float32(a + b)
    z = np.float32(s - a)
    return s, np.float32(np.float32(a - np.float32(s - z)) + np.float32(b - z))


def test_f64_triple_float_accumulation_is_float64_class():
    """The flush's triple-float accumulation (hi and lo by TwoSum, the errors
    and small into m2) of 400 chunk values with scales 2^0 .. 2^-40 equals
    their exact sum to 2^-53 of sum |c_k|: the only roundings are those of m2,
    whose magnitude stays near 2^-29 of the sum, against 400 * 2^-53 for a
    float64 summation of the same values."""
    rng = np.random.default_rng(31)
    m0 = m1 = m2 = np.float32(0.0)
    exact_sum = Fraction(0)
    total = Fraction(0)
    for k in range(400):
        hi = np.float32(rng.integers(-2 ** 22, 2 ** 22) / 2.0)          # multiple of 1/2 below 2^21
        lo = np.float32(rng.integers(-3 * 2 ** 22, 3 * 2 ** 22) * 2.0 ** -24)   # |lo| <= 3/4
        small = np.float32(rng.standard_normal() * 2.0 ** -10)
        sc = np.float32(2.0 ** -int(rng.integers(0, 41)))
        s0, e0 = two_sum_f32(m0, np.float32(hi * sc))
        s1, e1 = two_sum_f32(m1, np.float32(lo * sc))
        s2, e2 = two_sum_f32(s1, e0)
        m0, m1 = s0, s2
        m2 = np.float32(m2 + np.float32(np.float32(e1 + e2) + np.float32(small * sc)))
        c = (Fraction(float(hi)) + Fraction(float(lo)) + Fraction(float(small))) * Fraction(float(sc))
        exact_sum += c
        total += abs(c)
    got = Fraction(float(m0)) + Fraction(float(m1)) + Fraction(float(m2))
    assert abs(got - exact_sum) <= Fraction(1, 2 ** 53) * total


def f32_fixed(x, E0):
    """One float32 of the accumulator as an integer in units of
    2^(E0 - 187) (E0 the head's biased exponent): the mantissa shifted by
    E - E0 + 37, right shifts truncating toward zero on the magnitude."""
    b = int(np.float32(x).view(np.uint32))
    E = (b >> 23) & 255
    if E == 0:
        return 0
    M = (b & 0x7FFFFF) | 0x800000
    sh = E - E0 + 37
    v = M << sh if sh >= 0 else (M >> -sh if sh > -64 else 0)
    return -v if b >> 31 else v


def fixed_to_double(m0, m1, m2, e):
    """The epilogue's float64 of (m0 + m1 + m2) 2^e: the three floats as
    64-bit fixed-point integers aligned to the head, summed, rounded once to
    53 bits (nearest even), float64 fields assembled; None where the kernel
    takes its float64 path instead."""
    E0 = (int(np.float32(m0).view(np.uint32)) >> 23) & 255
    E1 = (int(np.float32(m1).view(np.uint32)) >> 23) & 255
    E2 = (int(np.float32(m2).view(np.uint32)) >> 23) & 255
    if E0 < 64 or E0 == 255 or E1 > E0 + 1 or E2 > E0 + 1 or E1 == 255 or E2 == 255:
        return None
    S = f32_fixed(m0, E0) + f32_fixed(m1, E0) + f32_fixed(m2, E0)
    assert -2 ** 63 < S < 2 ** 63
    if S == 0:
        return 0.0
    a = abs(S)
    sh = a.bit_length() - 53
    if sh > 0:
        mant = a >> sh
        rem, half = a & ((1 << sh) - 1), 1 << (sh - 1)
        if rem > half or (rem == half and mant & 1):
            mant += 1
        if mant >> 53:
            mant >>= 1
            sh += 1
    else:
        mant = a << -sh
    biased = sh + E0 - 187 + e + 52 + 1023
    if biased < 1 or biased > 2046:
        return None
    bits = (1 << 63 if S < 0 else 0) | (biased << 52) | (mant & ((1 << 52) - 1))
    return float(np.array(bits, dtype=np.uint64).view(np.float64))


def test_integer_float64_assembly_rounds_the_triple_float_once():
    """The product epilogue's conversion of the triple-float accumulator:
    on random accumulators (head, a tail up to 2^-20 below it and a smaller
    one, both signs, scales up to 2^+-900) the float64 it assembles is the
    exact sum m0 + m1 + m2 rounded to nearest, plus the bits that the fixed
    point drops (below one unit 2^(E0 - 187) <= 2^-60 |m0| for each of the
    two tails); special cases take the float64 path."""
    rng = np.random.default_rng(41)
    checked = 0
    for _ in range(3000):
        m0 = np.float32(rng.uniform(1, 2) * 2.0 ** int(rng.integers(-60, 60)) * rng.choice([-1, 1]))
        m1 = np.float32(float(m0) * rng.uniform(-1, 1) * 2.0 ** -int(rng.integers(0, 21)))
        m2 = np.float32(float(m1) * rng.uniform(-1, 1) * 2.0 ** -int(rng.integers(0, 30)))
        e = int(rng.integers(-900, 900))
        got = fixed_to_double(m0, m1, m2, e)
        if got is None:
            continue
        checked += 1
        exact = (Fraction(float(m0)) + Fraction(float(m1)) + Fraction(float(m2))) * Fraction(2) ** e
        ulp = Fraction(2) ** (math.frexp(float(exact))[1] - 53) if exact else Fraction(0)
        err = abs(Fraction(got) - exact)
        assert err <= ulp / 2 + Fraction(2) ** -59 * abs(Fraction(float(m0))) * Fraction(2) ** e, (m0, m1, m2, e)
    assert checked > 2500
    # the fall-back cases
    assert fixed_to_double(np.float32(0), np.float32(1), np.float32(0), 0) is None        # zero head
    assert fixed_to_double(np.float32(1), np.float32(8), np.float32(0), 0) is None        # tail above the head
    assert fixed_to_double(np.float32(np.inf), np.float32(0), np.float32(0), 0) is None   # non-finite
    assert fixed_to_double(np.float32(1), np.float32(0), np.float32(0), 1100) is None     # outside float64
    # exact cancellation to zero
    assert fixed_to_double(np.float32(1), np.float32(-1), np.float32(0), 0) == 0.0
