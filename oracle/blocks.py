"""Block primitives of the eigensolvers, in plain float64 (test oracle only).

Each function states the passage of arXiv:2409.05572 it follows.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# Relative pivot threshold below which a Cholesky factorisation of a Gram
# matrix is declared broken down (see ``cholesky_upper``).
CHOL_PIVOT_REL = 1e-14


def as_scipy(A):
    """Accept a workloads.CSR or a SciPy sparse matrix."""
    if sp.issparse(A):
        return A.tocsr()
    return sp.csr_matrix((A.data, A.indices, A.indptr), shape=(A.n, A.n))


def spmm(A, V: np.ndarray) -> np.ndarray:
    """Y = A V for sparse A and an n x w block V (the products A X, A W and
    A S of Algorithms 1-3)."""
    return np.asarray(as_scipy(A) @ V)


def gram(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """G = U^T V (the projected matrices X^T A X, S^T A S and the inner
    products of the orthogonalisation steps of Algorithms 1-3)."""
    return U.T @ V


def cholesky_upper(G: np.ndarray):
    """Textbook column Cholesky G = R^T R with R upper triangular.

    Returns (R, ok).  ok is False when a pivot d_j falls to or below
    CHOL_PIVOT_REL * G_jj (numerical rank loss), in which case R is None.
    """
    w = G.shape[0]
    R = np.zeros_like(G)
    for j in range(w):
        d = G[j, j] - R[:j, j] @ R[:j, j]
        if not (d > CHOL_PIVOT_REL * max(G[j, j], 0.0)) or not np.isfinite(d):
            return None, False
        rjj = np.sqrt(d)
        R[j, j] = rjj
        if j + 1 < w:
            R[j, j + 1:] = (G[j, j + 1:] - R[:j, j] @ R[:j, j + 1:]) / rjj
    return R, True


def cholqr_pass(W: np.ndarray):
    """One CholeskyQR pass W <- W R^{-1}, G = W^T W = R^T R.

    If the Cholesky factorisation breaks down, the shifted form of Fukaya,
    Kannan, Nakatsukasa, Yamamoto and Yanagisawa (SIAM J. Sci. Comput. 2020)
    is used: G + s I with s = 11 (m w + w (w + 1)) u ||W||_F^2.
    Returns (W_new, shifted).
    """
    m, w = W.shape
    if w == 0:
        return W.copy(), False
    G = gram(W, W)
    G = 0.5 * (G + G.T)
    R, ok = cholesky_upper(G)
    shifted = False
    if not ok:
        u = np.finfo(np.float64).eps / 2
        s = 11.0 * (m * w + w * (w + 1)) * u * float(np.trace(G))
        R, ok = cholesky_upper(G + s * np.eye(w))
        if not ok:
            raise np.linalg.LinAlgError("shifted CholeskyQR broke down")
        shifted = True
    Wn = sla.solve_triangular(R, W.T, trans="T", lower=False).T
    return Wn, shifted


def cholqr2(W: np.ndarray) -> np.ndarray:
    """The orthogonalisation step of Algorithms 1-3, for which the paper
    names no method: CholeskyQR2, i.e. two CholeskyQR passes; if the first pass needed the
    shift, a third pass follows (shifted CholeskyQR3)."""
    W1, shifted = cholqr_pass(W)
    if shifted:
        W1, _ = cholqr_pass(W1)
    W2, _ = cholqr_pass(W1)
    return W2


def orth_against(W: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """W <- W - Q (Q^T W) followed by orthogonalisation: Algorithm 3 projects
    the residual block out of span([X, P]) and then orthonormalises it; the
    expansion step treats S_drop against S the same way.

    Done twice (block classical Gram-Schmidt with reorthogonalisation, one
    CholeskyQR2 per pass) so that W is orthogonal to Q to working accuracy
    even when most of W lies in span(Q)."""
    for _ in range(2):
        if Q.shape[1] > 0:
            W = W - Q @ gram(Q, W)
        W = cholqr2(W)
    return W


def rayleigh_ritz(S: np.ndarray, AS: np.ndarray):
    """A_p = S^T A S (S orthonormal) and its spectral decomposition
    A_p = Z Lambda Z^T with Lambda ascending (Algorithms 1-3)."""
    Ap = gram(S, AS)
    Ap = 0.5 * (Ap + Ap.T)
    theta, Z = np.linalg.eigh(Ap)
    return theta, Z


def hl_trick(Z: np.ndarray, nnow: int, nlock: int):
    """Improved Hetmaniuk-Lehoucq basis selection (Algorithm 3; the paper
    defers the details to Duersch, Shao, Yang and Gu, SISC 2018, Sec. 4.2).

    S = [X, P, W] is orthonormal and Z holds all s eigenvectors of A_p.
    C_X = Z(:, 1:nnow) gives the new X.  The new P must be an orthonormal
    basis of span{X_new, X_old} orthogonal to X_new, restricted to the
    unlocked old columns nlock..nnow-1.  In coefficient space the old X is
    E = [I; 0]; its component orthogonal to C_X is Z_r Z_r^T E with
    Z_r = Z(:, nnow:s), so C_P = Z_r Q where Q is the orthonormal factor of
    the Householder QR of Z(nlock:nnow, nnow:s)^T.
    """
    CX = Z[:, :nnow]
    Zr = Z[:, nnow:]
    top = Zr[nlock:nnow, :]
    Q, _ = np.linalg.qr(top.T, mode="reduced")
    CP = Zr @ Q
    return CX, CP


def residual_test(X: np.ndarray, AX: np.ndarray, lam: np.ndarray,
                  normA: float, nev: int):
    """R = A X - X Lambda and the relative residual of Eq. conv per column,
    rho_i = ||r_i|| / (||A|| ||x_i|| + ||x_i|| |lambda_i|); the overall
    residual r^(j) of Eq. rk is the maximum over the first nev columns
    (Ritz values ascending)."""
    R = AX - X * lam[None, :]
    rn = np.linalg.norm(R, axis=0)
    xn = np.linalg.norm(X, axis=0)
    rho = rn / (normA * xn + xn * np.abs(lam))
    r = float(np.max(rho[:nev]))
    return R, rho, r


def cheb_filter(A, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """p_m(A) X with the scaled Chebyshev polynomial
    p_m(t) = T_m((t - c)/e) / T_m((a0 - c)/e), c = (a+b)/2, e = (b-a)/2,
    which damps [a, b] and equals 1 at a0 (Zhou and Saad's scaled three-term
    recurrence, SIMAX 2007, cited by the paper as Chebyshev-Davidson).
    Replaces the shift-and-invert solve of Algorithm 1."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma = e / (a0 - c)
    tau = 2.0 / sigma
    Y = (spmm(A, X) - c * X) * (sigma / e)
    Xp = X
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        Yn = (spmm(A, Y) - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * Xp
        Xp, Y, sigma = Y, Yn, sigma_new
    return Y
