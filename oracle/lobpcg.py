"""LOBPCG with soft locking and shrink-and-expand (arXiv:2409.05572,
Algorithm 3, inside the framework of Algorithm 5), in plain float64.

Notation follows the paper: X (n x nnow) Ritz vectors, P search directions,
W preconditioned residuals, S = [X, P, W], S_drop the columns dropped at the
last shrink, nex the initial/expanded width, nes the width after a shrink.

Readings (where the paper defers or is silent):
* "orthogonalize" is CholeskyQR2 (shifted CholeskyQR3 on breakdown), and
  projecting W against [X, P] (S_drop against S) is done twice.
* Soft locking: the locked columns are the longest leading run of the first
  nev Ritz pairs that satisfy Eq. conv.  A locked column stays in X and in
  the Rayleigh-Ritz step but gets no W column, and the P columns that belong
  to it are dropped.  P column t belongs to X column nlock + t.
* The improved Hetmaniuk-Lehoucq trick is ``blocks.hl_trick``.
* On a shrink S_drop = [X(:, nes:nnow), P(:, nes-nlock:)]: the tails of X and
  of P beyond column nes; on an expansion the first half of the
  re-orthogonalised S_drop is appended to X, the second half to P.
* Optional (not in the paper): a Jacobi preconditioner T = diag(A)^{-1} and
  deflation of a known null vector u0 (W, X0 kept orthogonal to u0).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import blocks as B
from .philox import gaussian_columns
from .strategy import Strategy


@dataclass
class Result:
    lam: np.ndarray
    X: np.ndarray
    converged: bool
    iters: int
    history: list = field(default_factory=list)      # r^(j), j = 1..iters
    widths: list = field(default_factory=list)       # nnow at the RR of each iteration
    events: list = field(default_factory=list)       # (j, "shrink"/"expand")
    rho: np.ndarray | None = None
    ritz: list = field(default_factory=list)         # per-iteration Ritz values (optional)


def _deflate(V, u0):
    if u0 is None:
        return V
    return V - np.outer(u0, u0 @ V)


def lobpcg(A, X0: np.ndarray, nev: int, nes: int, strategy: str = "none",
           tol: float = 1e-10, max_iter: int = 1000, normA: float = 1.0,
           precond: np.ndarray | None = None, u0: np.ndarray | None = None,
           keep_ritz: bool = False, observer=None, expand: str = "drop", seed: int = 0,
           **strategy_params) -> Result:
    """``observer(j, S, theta, X, P, expanded)``, if given, is called after
    the Rayleigh-Ritz step of every iteration (used by the invariant tests).

    ``expand``: "drop" appends the columns saved at the last shrink (S_drop);
    "random" (the 'Random' variant of Sec. 6.4) appends as many freshly drawn
    Gaussian columns instead (``philox.gaussian_columns`` with ``seed``, the
    e-th expansion of the solve drawing block e), treated exactly as S_drop
    would be."""
    n, nex = X0.shape
    assert nev <= nes < nex
    strat = Strategy(strategy, nes, nex, **strategy_params)

    # Algorithm 3 set-up: orthogonalise X0, Rayleigh-Ritz, X <- X Z.
    X = B.cholqr2(_deflate(X0, u0))
    AX = B.spmm(A, X)
    lam, Z = B.rayleigh_ritz(X, AX)
    X, AX = X @ Z, AX @ Z
    P = np.zeros((n, 0))
    AP = np.zeros((n, 0))
    nnow, nlock = nex, 0
    Sdrop = None
    n_exp = 0
    res = Result(lam[:nev], X[:, :nev], False, 0)

    for j in range(1, max_iter + 1):
        # R = AX - X Lambda; Eq. conv per column, Eq. rk overall.
        R, rho, r = B.residual_test(X, AX, lam, normA, nev)
        strat.record(j, r, float(rho[0]))
        res.history.append(r)
        res.iters = j
        if r <= tol:
            res.lam, res.X, res.converged, res.rho = lam[:nev].copy(), X[:, :nev].copy(), True, rho[:nev]
            break
        # Soft locking: deflate locked columns from P and R.
        conv = rho[:nev] <= tol
        new_lock = int(np.argmin(conv)) if not conv.all() else nev
        if new_lock > nlock:
            d = new_lock - nlock
            P, AP = P[:, d:], AP[:, d:]
        nlock = new_lock
        # W <- T R (unlocked columns), project against [X, P], orthogonalise.
        W = R[:, nlock:nnow]
        if precond is not None:
            W = W * precond[:, None]
        W = _deflate(W, u0)
        W = B.orth_against(W, np.hstack([X, P]))
        # Expansion: re-orthogonalise S_drop against S and split it.
        expanded = strat.ifexpand(j, nnow)
        if expanded:
            if expand == "random":
                Sdrop = _deflate(gaussian_columns(n, Sdrop.shape[1], seed, n_exp), u0)
            n_exp += 1
            S = np.hstack([X, P, W])
            Sd = B.orth_against(Sdrop, S)
            h = Sd.shape[1] // 2
            X = np.hstack([X, Sd[:, :h]])
            AX = np.hstack([AX, B.spmm(A, Sd[:, :h])])
            P = np.hstack([P, Sd[:, h:]])
            AP = np.hstack([AP, B.spmm(A, Sd[:, h:])])
            nnow = nex
        AW = B.spmm(A, W)
        S = np.hstack([X, P, W])
        AS = np.hstack([AX, AP, AW])
        theta, Z = B.rayleigh_ritz(S, AS)
        res.widths.append(nnow)
        if keep_ritz:
            res.ritz.append(theta[:nnow].copy())
        CX, CP = B.hl_trick(Z, nnow, nlock)
        X, AX = S @ CX, AS @ CX
        P, AP = S @ CP, AS @ CP
        lam = theta[:nnow]
        if observer is not None:
            observer(j, S, theta, X, P, expanded)
        if strat.ifshrink(j, nnow):
            q = nes - nlock
            Sdrop = np.hstack([X[:, nes:], P[:, q:]])
            X, AX, lam = X[:, :nes], AX[:, :nes], lam[:nes]
            P, AP = P[:, :q], AP[:, :q]
            nnow = nes
    else:
        res.lam, res.X = lam[:nev].copy(), X[:, :nev].copy()
        res.rho = B.residual_test(X, AX, lam, normA, nev)[1][:nev]
    res.events = list(strat.events)
    return res
