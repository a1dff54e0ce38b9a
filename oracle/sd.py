"""Steepest descent with shrink-and-expand (arXiv:2409.05572, Algorithm 2,
inside the framework of Algorithm 5), in plain float64.

Each iteration: R = AX - X Lambda, convergence test (Eq. conv / rk); on
expansion X <- [X, X_drop]; W = T R, W <- W - X (X^T W) and orthogonalise;
Rayleigh-Ritz on S = [X, W]; X <- S Z(:, 1:nnow); on shrink
X_drop <- X(:, nes+1:end), X <- X(:, 1:nes).  No locking (the paper locks only
in LOBPCG).

Reading: Algorithm 2 appends X_drop without re-orthogonalising it, but the
Rayleigh-Ritz step needs an orthonormal S; X_drop is orthogonalised against
the current X (twice, then CholeskyQR2) before it is appended.
"""
from __future__ import annotations

import numpy as np

from . import blocks as B
from .philox import gaussian_columns
from .lobpcg import Result
from .strategy import Strategy


def sd(A, X0: np.ndarray, nev: int, nes: int, strategy: str = "none", tol: float = 1e-10,
       max_iter: int = 1000, normA: float = 1.0, precond: np.ndarray | None = None,
       expand: str = "drop", seed: int = 0, **strategy_params) -> Result:
    """``expand`` = "random": fresh Gaussian columns (``philox.gaussian_columns``,
    block e at the e-th expansion) replace the saved X_drop, as for LOBPCG and
    subspace iteration (the 'Random' variant of Sec. 6.4)."""
    n, nex = X0.shape
    assert nev <= nes < nex
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
        if strat.ifexpand(j, nnow):
            if expand == "random":
                Xdrop = gaussian_columns(n, Xdrop.shape[1], seed, n_exp)
            n_exp += 1
            Xd = B.orth_against(Xdrop, X)
            X = np.hstack([X, Xd])
            AX = np.hstack([AX, B.spmm(A, Xd)])
            nnow = nex
        W = R if precond is None else R * precond[:, None]
        W = B.orth_against(W, X)
        S = np.hstack([X, W])
        AS = np.hstack([AX, B.spmm(A, W)])
        theta, Z = B.rayleigh_ritz(S, AS)
        res.widths.append(nnow)
        X, AX = S @ Z[:, :nnow], AS @ Z[:, :nnow]
        lam = theta[:nnow]
        if strat.ifshrink(j, nnow):
            Xdrop = X[:, nes:]
            X, AX, lam = X[:, :nes], AX[:, :nes], lam[:nes]
            nnow = nes
    else:
        res.lam, res.X = lam[:nev].copy(), X[:, :nev].copy()
        res.rho = B.residual_test(X, AX, lam, normA, nev)[1][:nev]
    res.events = list(strat.events)
    return res
