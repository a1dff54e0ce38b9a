"""Counter-based Gaussian columns for the 'Random' expansion of Sec. 6.4.

Test infrastructure (see oracle/__init__.py): the oracle's own
implementation of the published generator, shared with nothing.

The variant appends freshly drawn normally distributed columns at an
expansion instead of the saved X_drop.  Both sides of the parity tests draw
them from one definition, so that the draws need not be passed in:

* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11): a 128-bit counter (c0, c1, c2, c3) and a 64-bit
  key (k0, k1); ten rounds of
      (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2   (32 x 32 -> 64 bits)
      (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key bumped by the Weyl constants
  (0x9E3779B9, 0xBB67AE85) after every round but the last.
* Entry (i, j) of the block drawn at the e-th expansion of a solve with
  seed s: counter (i mod 2^32, floor(i / 2^32), floor(j / 2), e), key
  (s mod 2^32, floor(s / 2^32)); output words w0..w3 give the float64
  uniforms u1 = (w0 2^21 + floor(w1 / 2^11) + 1/2) 2^-53 in (0, 1) and
  u2 = (w2 2^21 + floor(w3 / 2^11)) 2^-53 in [0, 1); Box-Muller:
  z = sqrt(-2 ln u1) cos(2 pi u2) for even j, sqrt(-2 ln u1) sin(2 pi u2)
  for odd j.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of counters (uint64 arrays holding 32-bit
    values) with one key; returns the four output words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0, k1 = np.uint64(k0 & MASK), np.uint64(k1 & MASK)
    for rnd in range(10):
        p0 = c0 * np.uint64(M0)            # < 2^64: exact in uint64
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return c0, c1, c2, c3


def gaussian_columns(n: int, w: int, seed: int, e: int) -> np.ndarray:
    """The n x w block of the e-th expansion (module docstring)."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(w, dtype=np.uint64)[None, :]
    i, j = np.broadcast_arrays(i, j)
    w0, w1, w2, w3 = philox4x32_10(i & np.uint64(MASK), i >> np.uint64(32), j >> np.uint64(1),
                                   np.full(i.shape, e, dtype=np.uint64), seed & MASK, seed >> 32)
    t = 2.0 ** -53
    u1 = ((w0.astype(np.float64) * 2.0 ** 21 + (w1 >> np.uint64(11)).astype(np.float64)) + 0.5) * t
    u2 = (w2.astype(np.float64) * 2.0 ** 21 + (w3 >> np.uint64(11)).astype(np.float64)) * t
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return np.where((j & np.uint64(1)) == 0, r * np.cos(ang), r * np.sin(ang))
