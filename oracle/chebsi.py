"""Subspace iteration with shrink-and-expand (arXiv:2409.05572, Algorithm 1,
inside the framework of Algorithm 5), in plain float64.

The shift-and-invert step X <- (A - zeta I)^{-1} X is replaced by a degree-m
Chebyshev filter X <- p_m(A) X (``blocks.cheb_filter``); the theory of the
paper's Sec. 5 is stated for a power step X <- B X, which p_m(A) is.

Readings: Ritz values are sorted algebraically ascending (the Anderson
Hamiltonian is indefinite, so an ordering by magnitude would pick interior
eigenvalues); the filter damps [a, b] with a = the largest Ritz value of the
active block, b = an upper bound on the spectrum supplied by the caller,
scaled to 1 at a0 = the smallest Ritz value.
"""
from __future__ import annotations

import numpy as np

from . import blocks as B
from .philox import gaussian_columns
from .lobpcg import Result
from .strategy import Strategy


def chebsi(A, X0: np.ndarray, nev: int, nes: int, strategy: str = "none",
           tol: float = 1e-10, max_iter: int = 1000, normA: float = 1.0,
           degree: int = 12, upper: float | None = None,
           keep_ritz: bool = False, expand: str = "drop", observer=None, seed: int = 0,
           **strategy_params) -> Result:
    """``expand``: "drop" appends the columns dropped at the last shrink;
    "powered" (the powered X_drop variant of Sec. 6.4) also applies the iteration's
    operator -- here the same Chebyshev filter -- to the saved columns every
    iteration, without orthogonalising them; "random" (the 'Random' variant)
    appends freshly drawn Gaussian columns (``philox.gaussian_columns`` with
    ``seed``, block e at the e-th expansion) instead of the saved ones.

    ``observer(j, lam, nnow, drop_before, drop_after)``, if given, is called
    after the filter step of iteration j with the Ritz values the filter was
    built from, the active width, and copies of the saved columns before and
    after that step (None while nothing is saved)."""
    n, nex = X0.shape
    assert nev <= nes < nex
    if upper is None:
        upper = normA
    strat = Strategy(strategy, nes, nex, **strategy_params)

    X = B.cholqr2(X0)
    AX = B.spmm(A, X)
    lam, Z = B.rayleigh_ritz(X, AX)
    X, AX = X @ Z, AX @ Z
    nnow = nex
    Xdrop = None
    n_exp = 0
    res = Result(lam[:nev], X[:, :nev], False, 0)

    for j in range(1, max_iter + 1):
        R, rho, r = B.residual_test(X, AX, lam, normA, nev)
        strat.record(j, r, float(rho[0]))
        res.history.append(r)
        res.iters = j
        if r <= tol:
            res.lam, res.X, res.converged, res.rho = lam[:nev].copy(), X[:, :nev].copy(), True, rho[:nev]
            break
        # X <- p_m(A) X replaces X <- (A - zeta I)^{-1} X.
        a, a0 = float(lam[nnow - 1]), float(lam[0])
        X = B.cheb_filter(A, X, degree, a, upper, a0)
        before = None if (observer is None or Xdrop is None) else Xdrop.copy()
        if expand == "powered" and Xdrop is not None:
            Xdrop = B.cheb_filter(A, Xdrop, degree, a, upper, a0)
        if observer is not None:
            observer(j, lam.copy(), nnow, before, None if Xdrop is None else Xdrop.copy())
        if strat.ifexpand(j, nnow):
            if expand == "random":
                Xdrop = gaussian_columns(n, Xdrop.shape[1], seed, n_exp)
            n_exp += 1
            X = np.hstack([X, Xdrop])
            nnow = nex
        X = B.cholqr2(X)
        AX = B.spmm(A, X)
        lam, Z = B.rayleigh_ritz(X, AX)
        X, AX = X @ Z, AX @ Z
        res.widths.append(nnow)
        if keep_ritz:
            res.ritz.append(lam.copy())
        if strat.ifshrink(j, nnow):
            Xdrop = X[:, nes:]
            X, AX, lam = X[:, :nes], AX[:, :nes], lam[:nes]
            nnow = nes
    else:
        res.lam, res.X = lam[:nev].copy(), X[:, :nev].copy()
        res.rho = B.residual_test(X, AX, lam, normA, nev)[1][:nev]
    res.events = list(strat.events)
    return res
