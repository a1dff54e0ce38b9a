"""Shrink-and-expand strategies (arXiv:2409.05572, Sec. 3.2, Algorithms 6
and 7, Eqs. ckslope and ckslopek, and the warm-up rule that closes Sec. 3.2).

Readings taken where the paper is silent or garbled:

* r^(j) is the residual of Eq. rk computed at the start of iteration j; the
  slope of Eq. ckslope exists for j >= 2, that of Eq. ckslopek for j > jp.
* Warm-up: no decision is taken until the first shrink, which happens at the
  first iteration j with j >= j_warm and r^(j) <= r_warm (call it j0).
* fix: Algorithm 6 uses the absolute iteration count, which would disagree
  with the warm-up; its clock is started at the first shrink, j' = j - j0 + js,
  so an expansion happens when mod(j - j0 + js, je) = 0 and nnow = nes, and a
  shrink when mod(j - j0, je) = 0 and nnow > nes (js iterations after each
  expansion).
* slope/slopek shrink: the condition printed in Algorithm 7 compares j_l
  with j_e, while the text ties the shrink to a fixed js after each
  expansion; the shrink fires when j_l = js, j_l counting iterations since
  the last expansion.
* slope/slopek expand: Algorithm 7's test c_max / c > mu misbehaves for
  c <= 0, while the text expands when the residual grows; the test used is
  mu * c < c_max (same as c_max/c > mu for c > 0), with c_max the largest slope
  since the last shrink including the current iteration's slope.
* A shrink only happens when nnow > nes (it would be a no-op otherwise).
* Aggressive warm-up (closing remarks of the paper): with warm_first the
  gate compares the residual of the first Ritz pair, instead of r^(j) (in
  practice the nev-th pair's), with r_warm; the paper pairs it with
  r_warm = 1e-1.
"""
from __future__ import annotations

import math

NONE, FIX, SLOPE, SLOPEK = "none", "fix", "slope", "slopek"
KINDS = (NONE, FIX, SLOPE, SLOPEK)


class Strategy:
    def __init__(self, kind: str, nes: int, nex: int, je: int = 12, js: int = 2,
                 mu: float = 1.1, jp: int = 10, j_warm: int = 5, r_warm: float = 1e-4,
                 warm_first: bool = False):
        if kind not in KINDS:
            raise ValueError(kind)
        self.kind, self.nes, self.nex = kind, nes, nex
        self.je, self.js, self.mu, self.jp = je, js, mu, jp
        self.j_warm, self.r_warm = j_warm, r_warm
        self.warm_first = bool(warm_first)
        self.r = {}            # j -> r^(j)
        self.r1 = {}           # j -> Eq. conv residual of the first Ritz pair
        self.warmed = False
        self.j0 = None         # iteration of the first shrink
        self.j_exp = None      # iteration of the last expansion
        self.c_max = None      # largest slope since the last shrink
        self.events = []       # (j, "shrink" | "expand")

    # -- Eq. rk history -------------------------------------------------
    def record(self, j: int, r: float, r1: float | None = None) -> None:
        self.r[j] = r
        self.r1[j] = r if r1 is None else r1

    @staticmethod
    def _log10(x: float) -> float:
        return math.log10(max(x, 1e-300))

    def slope(self, j: int):
        """c^(j) of Eq. ckslope (slope) or Eq. ckslopek (slopek)."""
        if self.kind == SLOPE:
            if (j - 1) not in self.r:
                return None
            return self._log10(self.r[j - 1]) - self._log10(self.r[j])
        if self.kind == SLOPEK:
            if j < self.jp or (j - self.jp) not in self.r:
                return None
            return (self._log10(self.r[j - self.jp]) - self._log10(self.r[j])) / self.jp
        return None

    # -- Algorithms 6 / 7 -----------------------------------------------
    def ifexpand(self, j: int, nnow: int) -> bool:
        if self.kind == NONE or not self.warmed:
            return False
        if self.kind == FIX:
            go = nnow == self.nes and (j - self.j0 + self.js) % self.je == 0
        else:
            c = self.slope(j)
            if c is None or nnow != self.nes:
                go = False
            else:
                self.c_max = c if self.c_max is None else max(self.c_max, c)
                go = self.mu * c < self.c_max
        if go:
            self.j_exp = j
            self.events.append((j, "expand"))
        return go

    def ifshrink(self, j: int, nnow: int) -> bool:
        if self.kind == NONE or nnow <= self.nes:
            return False
        if not self.warmed:
            gate = self.r1[j] if self.warm_first else self.r[j]
            go = j >= self.j_warm and gate <= self.r_warm
            if go:
                self.warmed = True
                self.j0 = j
        elif self.kind == FIX:
            go = (j - self.j0) % self.je == 0
        else:
            go = self.j_exp is not None and (j - self.j_exp) == self.js
        if go:
            self.c_max = None
            self.events.append((j, "shrink"))
        return go
