"""Pins of the FP64 oracle against what the paper and the mathematics fix:
closed-form spectra, brute force, the paper's printed 3x3 example,
Prop. 1 and Thm. 1, invariants and special cases.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import blocks as B
from oracle.chebsi import chebsi
from oracle.lobpcg import lobpcg
from paper_2409_05572_gb300 import workloads as W


# ---------------------------------------------------------------------------
# helpers written in the tests (independent of the oracle)
# ---------------------------------------------------------------------------
def jacobi_eigvals(M, sweeps=60):
    """Textbook cyclic Jacobi eigenvalue iteration (brute force, dense)."""
    A = np.array(M, dtype=np.float64)
    n = A.shape[0]
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.tril(A, -1) ** 2))
        if off < 1e-15 * np.linalg.norm(A):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(A[p, q]) < 1e-300:
                    continue
                tau = (A[q, q] - A[p, p]) / (2 * A[p, q])
                t = math.copysign(1.0, tau) / (abs(tau) + math.sqrt(1 + tau * tau))
                c = 1 / math.sqrt(1 + t * t)
                s = t * c
                Ap, Aq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * Ap - s * Aq, s * Ap + c * Aq
                Ap, Aq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * Ap - s * Aq, s * Ap + c * Aq
    return np.sort(np.diag(A))


def dirichlet_spectrum(dims):
    axes = [4 * np.sin(np.arange(1, d + 1) * np.pi / (2 * (d + 1))) ** 2 for d in dims]
    tot = axes[0]
    for a in axes[1:]:
        tot = np.add.outer(tot, a).ravel()
    return np.sort(tot)


def subspace_dist(U, V):
    """|| U U^T - V V^T ||_2 for orthonormal U, V."""
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    return np.linalg.norm(Qu @ Qu.T - Qv @ Qv.T, 2)


def load_golden(path):
    vals = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        vals[k] = np.array([float(x) for x in v])
    return vals


# ---------------------------------------------------------------------------
# workloads (inputs) against closed forms
# ---------------------------------------------------------------------------
def test_laplacian_generators_match_closed_form():
    for dims, gen in (((7, 5), lambda: W.laplacian_2d(7, 5)),
                      ((4, 3, 5), lambda: W.laplacian_3d(4, 3, 5))):
        A = gen().to_scipy().toarray()
        assert np.allclose(A, A.T)
        assert np.allclose(np.linalg.eigvalsh(A), dirichlet_spectrum(dims), atol=1e-12)
        assert abs(W.dirichlet_norm(dims) - dirichlet_spectrum(dims)[-1]) < 1e-12


def test_c1_c2_closed_form_values():
    # Values quoted for the 32x32 and 128^3 grids (c1 and c2 workloads).
    ev = dirichlet_spectrum((32, 32))[:11]
    assert np.allclose(ev[:10], [0.0181123, 0.0451988, 0.0451988, 0.0722852, 0.0900702,
                                 0.0900702, 0.1171567, 0.1171567, 0.1523203, 0.1523203],
                       atol=5e-8)
    assert abs(ev[10] - 0.16203) < 1e-5
    d = 4 * np.sin(np.arange(1, 8) * np.pi / 258) ** 2
    tot = np.sort(np.add.outer(np.add.outer(d, d), d).ravel())
    assert abs(tot[0] - 0.00177918) < 1e-8
    assert abs(tot[63] - 0.01955692) < 1e-8


def test_anderson_zero_disorder_is_periodic_closed_form():
    L = 6
    A = W.anderson_3d(L, disorder=0.0).to_scipy().toarray()
    c = -2 * np.cos(2 * np.pi * np.arange(L) / L)
    ex = np.sort(np.add.outer(np.add.outer(c, c), c).ravel())
    assert np.allclose(np.linalg.eigvalsh(A), ex, atol=1e-12)
    assert abs(ex[0] + 6.0) < 1e-12


def test_anderson_disorder_range_and_structure():
    A = W.anderson_3d(10, seed=2)
    M = A.to_scipy()
    d = M.diagonal()
    assert A.n == 1000 and A.nnz == 7000
    assert d.min() >= -8.25 and d.max() <= 8.25
    assert abs((M - M.T)).max() == 0
    assert W.gershgorin_bound(A) <= 8.25 + 6 + 1e-12


def test_graph_laplacian_null_vector_and_symmetry():
    A = W.graph_laplacian(3000, seed=3)
    M = A.to_scipy()
    assert abs(M @ np.ones(A.n)).max() < 1e-10
    assert abs(M - M.T).max() < 1e-14
    off = -M.copy()
    off.setdiag(0)
    off.eliminate_zeros()
    assert off.data.min() >= 0.5 - 1e-12
    deg = np.diff(M.indptr) - 1
    assert 8.0 < deg.mean() < 12.0
    # connected: exactly one zero eigenvalue
    ev = np.linalg.eigvalsh(M.toarray())
    assert abs(ev[0]) < 1e-10 and ev[1] > 1e-8


def test_ring_graph_laplacian_closed_form_through_spmm():
    n, w = 40, 0.75
    i = np.arange(n)
    rows = np.concatenate([i, i, i])
    cols = np.concatenate([i, (i + 1) % n, (i - 1) % n])
    vals = np.concatenate([np.full(n, 2 * w), np.full(n, -w), np.full(n, -w)])
    L = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    m = 3
    v = np.cos(2 * np.pi * m * i / n)
    lam = 2 * w * (1 - np.cos(2 * np.pi * m / n))
    assert np.allclose(B.spmm(L, v[:, None])[:, 0], lam * v, atol=1e-13)


def test_norm_estimate_is_tight_lower_bound():
    A = W.laplacian_2d(12)
    est = W.norm_estimate(A)
    true = dirichlet_spectrum((12, 12))[-1]
    assert est <= true + 1e-12 and est > true * 0.999


# ---------------------------------------------------------------------------
# block primitives
# ---------------------------------------------------------------------------
def test_spmm_brute_force():
    rng = np.random.default_rng(5)
    M = sp.random(37, 37, density=0.2, random_state=5, format="csr")
    V = rng.standard_normal((37, 6))
    D = M.toarray()
    ref = np.array([[sum(D[i, k] * V[k, j] for k in range(37)) for j in range(6)]
                    for i in range(37)])
    assert np.allclose(B.spmm(M, V), ref, atol=1e-13)


def test_gram_is_not_transposed():
    U = np.arange(6.0).reshape(3, 2)
    V = np.arange(9.0).reshape(3, 3)
    G = B.gram(U, V)
    assert G.shape == (2, 3)
    assert G[1, 2] == sum(U[i, 1] * V[i, 2] for i in range(3))


def test_cholesky_upper_against_definition():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((30, 8))
    G = Y.T @ Y
    R, ok = B.cholesky_upper(G)
    assert ok
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(R.T @ R, G, rtol=1e-13, atol=1e-12)
    G2 = G.copy()
    G2[:, 3] = G2[:, 2]
    G2[3, :] = G2[2, :]
    _, ok2 = B.cholesky_upper(G2)
    assert not ok2


def test_cholqr2_orthonormal_and_same_span():
    rng = np.random.default_rng(2)
    Wm = rng.standard_normal((500, 12))
    Q = B.cholqr2(Wm)
    assert np.linalg.norm(Q.T @ Q - np.eye(12)) < 1e-13
    # Q R = W with R = Q^T W upper triangular and positive diagonal
    R = Q.T @ Wm
    assert np.linalg.norm(np.tril(R, -1)) < 1e-12 * np.linalg.norm(R)
    assert np.all(np.diag(R) > 0)
    assert np.linalg.norm(Q @ R - Wm) < 1e-12 * np.linalg.norm(Wm)


def test_cholqr2_ill_conditioned_takes_shifted_path():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((400, 10)))
    V, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    Wm = U @ np.diag(np.logspace(0, -11, 10)) @ V.T
    _, shifted = B.cholqr_pass(Wm)
    assert shifted
    Q = B.cholqr2(Wm)
    assert np.linalg.norm(Q.T @ Q - np.eye(10)) < 1e-12


def test_orth_against_removes_span():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((300, 9)))
    Wm = Q @ rng.standard_normal((9, 5)) + 1e-9 * rng.standard_normal((300, 5))
    Wo = B.orth_against(Wm, Q)
    assert np.linalg.norm(Q.T @ Wo) < 1e-13
    assert np.linalg.norm(Wo.T @ Wo - np.eye(5)) < 1e-13


def test_rayleigh_ritz_exact_on_invariant_subspace():
    rng = np.random.default_rng(6)
    d = np.sort(rng.uniform(1, 9, 40))
    Qf, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    A = Qf @ np.diag(d) @ Qf.T
    S = Qf[:, [5, 1, 7]] @ np.linalg.qr(rng.standard_normal((3, 3)))[0]
    theta, Z = B.rayleigh_ritz(S, A @ S)
    assert np.allclose(theta, np.sort(d[[1, 5, 7]]), atol=1e-13)
    assert np.all(np.diff(theta) >= 0)


def test_residual_test_eq_conv_by_hand():
    X = np.array([[1.0, 0.0], [0.0, 2.0], [0.0, 0.0]])
    AX = np.array([[2.0, 0.0], [0.0, 6.0], [0.5, 0.0]])
    lam = np.array([2.0, 3.0])
    normA = 10.0
    R, rho, r = B.residual_test(X, AX, lam, normA, nev=1)
    assert np.allclose(R, [[0, 0], [0, 0], [0.5, 0]])
    assert abs(rho[0] - 0.5 / (10 * 1 + 1 * 2)) < 1e-16
    assert rho[1] == 0.0
    assert r == rho[0]


def test_hl_trick_spans_old_and_new_x():
    rng = np.random.default_rng(7)
    s, nnow, nlock = 30, 10, 3
    M = rng.standard_normal((s, s))
    M = M + M.T
    _, Z = np.linalg.eigh(M)
    CX, CP = B.hl_trick(Z, nnow, nlock)
    assert CP.shape == (s, nnow - nlock)
    assert np.linalg.norm(CP.T @ CP - np.eye(nnow - nlock)) < 1e-13
    assert np.linalg.norm(CX.T @ CP) < 1e-13
    E = np.eye(s)[:, nlock:nnow]
    # old active X columns lie in span{C_X, C_P}
    basis = np.hstack([CX, CP])
    assert np.linalg.norm(E - basis @ (basis.T @ E)) < 1e-12
    # and nothing else: C_P lies in span{C_X, E}
    sp2 = np.linalg.qr(np.hstack([CX, E]))[0]
    assert np.linalg.norm(CP - sp2 @ (sp2.T @ CP)) < 1e-12


# ---------------------------------------------------------------------------
# Chebyshev filter: p(A) v = p(lambda) v, p = scaled T_m
# ---------------------------------------------------------------------------
def _cheb_T(m, x):
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def test_cheb_filter_closed_form():
    lam = np.array([-3.0, -2.5, -1.0, 0.5, 2.0, 4.0, 7.5, 9.0])
    A = sp.diags(lam).tocsr()
    V = np.eye(8)
    m, a, b, a0 = 12, -0.5, 9.0, -3.0
    Y = B.cheb_filter(A, V, m, a, b, a0)
    c, e = (a + b) / 2, (b - a) / 2
    p = _cheb_T(m, (lam - c) / e) / _cheb_T(m, np.array([(a0 - c) / e]))[0]
    assert np.allclose(np.diag(Y), p, rtol=1e-12, atol=1e-14)
    assert abs(np.diag(Y)[0] - 1.0) < 1e-12
    assert np.abs(np.diag(Y)[4:]).max() <= 1.0 / abs(_cheb_T(m, np.array([(a0 - c) / e]))[0]) + 1e-15


# ---------------------------------------------------------------------------
# The paper's 3x3 example (Sec. 4), Prop. 1 and Thm. 1
# ---------------------------------------------------------------------------
def _prop1_rate(A, x, v1, lam1):
    xc = x - v1 * (v1 @ x)
    xc /= np.linalg.norm(xc)
    return lam1 * np.linalg.norm(np.linalg.solve(A, xc))


def _match_up_to_sign(X, ref, rtol):
    for j in range(X.shape[1]):
        s = np.sign(X[np.argmax(np.abs(ref[:, j])), j]) * np.sign(ref[np.argmax(np.abs(ref[:, j])), j])
        assert np.allclose(s * X[:, j], ref[:, j], rtol=rtol, atol=5e-5 * np.abs(ref[:, j]).max()), (X, ref)


def test_worked_example_si_step(golden_dir):
    g = load_golden(os.path.join(golden_dir, "worked_example_3x3.txt"))
    A = np.diag(g["A_diag"])
    X0 = g["X0"].reshape(3, 2)
    X = B.cholqr2(X0)
    _, Z = B.rayleigh_ritz(X, A @ X)
    X = X @ Z
    X = np.linalg.solve(A, X)
    X = B.cholqr2(X)
    _, Z = B.rayleigh_ritz(X, A @ X)
    X1 = X @ Z
    _match_up_to_sign(X1, g["X1"].reshape(3, 2), 1e-4)
    rho = _prop1_rate(A, X1[:, 0], np.eye(3)[:, 0], 1.0)
    assert abs(rho - g["rho1"][0]) < 1e-6


def test_worked_example_expansion(golden_dir):
    g = load_golden(os.path.join(golden_dir, "worked_example_3x3.txt"))
    A = np.diag(g["A_diag"])
    X0 = g["X0"].reshape(3, 2)
    x = np.linalg.solve(A, X0[:, :1])
    x = B.cholqr2(x)
    assert np.allclose(np.abs(x[:, 0]) * math.sqrt(10101), [100, 10, 1])
    rho_b = _prop1_rate(A, x[:, 0], np.eye(3)[:, 0], 1.0)
    assert abs(rho_b - g["rho_before"][0]) < 5e-5
    # expansion: append X0's second column, then apply the operator to the
    # expanded block (the reading that reproduces the printed numbers)
    Xe = np.hstack([x, X0[:, 1:]])
    X = B.cholqr2(np.linalg.solve(A, Xe))
    _, Z = B.rayleigh_ritz(X, A @ X)
    X2 = X @ Z
    _match_up_to_sign(X2, g["X2"].reshape(3, 2), 1e-4)
    rho2 = _prop1_rate(A, X2[:, 0], np.eye(3)[:, 0], 1.0)
    assert abs(rho2 - g["rho2"][0]) < 1e-6
    assert rho2 < 0.5 * 0.1 < rho_b


def test_prop1_rate_matches_tangent_ratio():
    rng = np.random.default_rng(8)
    d = np.array([1.0, 3.0, 4.0, 9.0, 20.0])
    A = np.diag(d)
    x = rng.standard_normal(5)
    v1 = np.eye(5)[:, 0]
    tan0 = np.linalg.norm(x - v1 * x[0]) / abs(x[0])
    y = B.cholqr2(np.linalg.solve(A, x)[:, None])[:, 0]
    tan1 = np.linalg.norm(y - v1 * y[0]) / abs(y[0])
    assert abs(tan1 / tan0 - _prop1_rate(A, x / np.linalg.norm(x), v1, 1.0)) < 1e-12


def test_thm1_rate_bound_on_diagonal_B():
    rng = np.random.default_rng(9)
    n, k, l = 60, 4, 9
    sig = np.sort(rng.uniform(0.1, 10.0, n))[::-1]
    Bm = np.diag(sig)
    for _ in range(20):
        X = B.cholqr2(rng.standard_normal((n, k)))
        Xk, Xlk, Xperp = X[:k], X[k:l], X[l:]
        Xki = np.linalg.inv(Xk)

        def tan_angle(Y):
            Q = B.cholqr2(Y)
            cosm = np.linalg.svd(Q[:k], compute_uv=False).min()
            return math.sqrt(max(1 - cosm ** 2, 0)) / cosm

        lhs = tan_angle(Bm @ X) / tan_angle(X)
        ratio = np.linalg.norm(Xlk @ Xki, 2) / np.linalg.norm(np.vstack([Xlk, Xperp]) @ Xki, 2)
        rhs = sig[l] / sig[k - 1] + (sig[k] - sig[l]) / sig[k - 1] * ratio
        assert lhs <= rhs * (1 + 1e-10)


# ---------------------------------------------------------------------------
# whole solvers
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1():
    A = W.laplacian_2d(32)
    return A, W.dirichlet_norm((32, 32)), W.gaussian_block(A.n, 20, 0), dirichlet_spectrum((32, 32))


@pytest.mark.parametrize("strategy", ["none", "fix", "slope", "slopek"])
def test_c1_lobpcg_matches_closed_form(c1, strategy):
    A, normA, X0, ex = c1
    r = lobpcg(A, X0, 10, 15, strategy, tol=1e-10, normA=normA)
    assert r.converged
    assert np.max(np.abs(r.lam - ex[:10]) / ex[:10]) < 1e-12
    M = A.to_scipy()
    res = np.linalg.norm(M @ r.X - r.X * r.lam, axis=0) / normA
    assert res.max() <= 2e-10
    assert np.linalg.norm(r.X.T @ r.X - np.eye(10)) < 1e-12
    if strategy != "none":
        assert any(e == "shrink" for _, e in r.events)
        assert any(e == "expand" for _, e in r.events)
        assert min(r.widths) == 15 and max(r.widths) == 20


def test_lobpcg_invariants_every_iteration(c1):
    A, normA, X0, ex = c1
    M = A.to_scipy()
    prev = {}

    def obs(j, S, theta, X, P, expanded):
        s = S.shape[1]
        assert np.linalg.norm(S.T @ S - np.eye(s)) < 1e-11
        XP = np.hstack([X, P])
        assert np.linalg.norm(XP.T @ XP - np.eye(XP.shape[1])) < 1e-11
        # Cauchy interlacing against the closed-form spectrum
        n = A.n
        for i in range(s):
            assert ex[i] - 1e-12 <= theta[i] <= ex[n - s + i] + 1e-12
        nn = X.shape[1]
        if "theta" in prev and not expanded:
            m = min(nn, len(prev["theta"]))
            assert np.all(theta[:m] <= prev["theta"][:m] + 1e-12)
        prev["theta"] = theta[:nn].copy()

    r = lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA, observer=obs)
    assert r.converged


def test_lobpcg_jacobi_precond_and_deflation_graph():
    A = W.graph_laplacian(600, seed=3)
    M = A.to_scipy()
    ev = np.linalg.eigvalsh(M.toarray())
    u0 = np.ones(A.n) / math.sqrt(A.n)
    X0 = W.gaussian_block(A.n, 16, 3)
    normA = float(ev[-1])
    r = lobpcg(A, X0, 8, 11, "fix", tol=1e-9, normA=normA, precond=1.0 / M.diagonal(), u0=u0,
               max_iter=600)
    assert r.converged
    assert np.max(np.abs(r.lam - ev[1:9]) / ev[1:9]) < 1e-9
    assert np.abs(u0 @ r.X).max() < 1e-10


def test_lobpcg_brute_force_random_spd():
    rng = np.random.default_rng(10)
    n = 80
    M = sp.random(n, n, density=0.08, random_state=10)
    M = (M + M.T + sp.diags(rng.uniform(0.5, 3.0, n) + 4.0)).tocsr()
    ev = jacobi_eigvals(M.toarray())
    X0 = W.gaussian_block(n, 12, 10)
    r = lobpcg(M, X0, 6, 8, "slope", tol=1e-11, normA=float(ev[-1]), j_warm=2, r_warm=1e-2)
    assert r.converged
    assert np.allclose(r.lam, ev[:6], rtol=1e-10)


def test_lobpcg_none_vs_scipy_lobpcg():
    from scipy.sparse.linalg import lobpcg as sp_lobpcg
    A = W.laplacian_2d(20)
    M = A.to_scipy()
    X0 = W.gaussian_block(A.n, 12, 12)
    ours = lobpcg(A, X0, 6, 8, "none", tol=1e-10, normA=W.dirichlet_norm((20, 20)))
    lam, _ = sp_lobpcg(M, X0.copy(), largest=False, tol=1e-9, maxiter=500)
    assert np.allclose(ours.lam, np.sort(lam)[:6], rtol=1e-9)


def test_chebsi_anderson_brute_force():
    A = W.anderson_3d(6, seed=2)
    ev = jacobi_eigvals(A.to_scipy().toarray(), sweeps=30)
    X0 = W.gaussian_block(A.n, 16, 2)
    ub = W.gershgorin_bound(A)
    for strat in ("none", "fix", "slopek"):
        r = chebsi(A, X0, 8, 11, strat, tol=1e-11, normA=float(np.abs(ev).max()), degree=8,
                   upper=ub, j_warm=2, r_warm=1e-2, je=4, js=1, jp=2)
        assert r.converged
        assert np.allclose(r.lam, ev[:8], rtol=1e-10, atol=1e-12)


def test_chebsi_c1_shrinks_and_matches():
    A = W.laplacian_2d(32)
    ex = dirichlet_spectrum((32, 32))
    X0 = W.gaussian_block(A.n, 20, 0)
    r = chebsi(A, X0, 10, 15, "fix", tol=1e-11, normA=W.dirichlet_norm((32, 32)), degree=12,
               upper=8.0, j_warm=2, r_warm=1e-1, je=3, js=1)
    assert r.converged
    assert np.allclose(r.lam, ex[:10], rtol=1e-12)
    assert any(e == "shrink" for _, e in r.events)


# ---------------------------------------------------------------------------
# Algorithm 2 (SD) and the powered X_drop expansion (Sec. 6.4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("strategy", ["none", "fix", "slopek"])
def test_sd_matches_closed_form(strategy):
    from oracle.sd import sd
    A = W.laplacian_2d(16, 12)
    ex = dirichlet_spectrum((16, 12))
    X0 = W.gaussian_block(A.n, 12, 5)
    r = sd(A, X0, 6, 8, strategy, tol=1e-10, normA=W.dirichlet_norm((16, 12)), max_iter=3000,
           j_warm=3, r_warm=1e-3, je=6, js=1, jp=3)
    assert r.converged
    assert np.allclose(r.lam, ex[:6], rtol=1e-11)
    if strategy != "none":
        assert any(e == "expand" for _, e in r.events)


@pytest.mark.parametrize("expand", ["powered", "drop"])
def test_chebsi_powered_drop_step_closed_form(expand):
    """Sec. 6.4, powered X_drop: on a diagonal A every saved column is
    multiplied, once per iteration, by the filter p_m(d_i) of that iteration
    (the closed form T_m((d - c)/e) / T_m((a0 - c)/e) with a, a0 the largest
    active and the smallest Ritz value); the plain variant leaves the saved
    columns untouched.  Between two shrinks the saved block of an iteration is
    the previous iteration's result, so the product of the filters is applied
    without orthogonalisation."""
    rng = np.random.default_rng(7)
    d = np.sort(rng.uniform(0.0, 10.0, 60))
    A = W.CSR(60, np.arange(61, dtype=np.int32), np.arange(60, dtype=np.int32), d)
    X0 = rng.standard_normal((60, 12))
    seen = []
    r = chebsi(A, X0, 4, 8, "fix", tol=1e-12, normA=10.0, degree=6, upper=10.5, max_iter=40,
               j_warm=2, r_warm=1e-1, je=5, js=1, expand=expand,
               observer=lambda *a: seen.append(a))
    shrinks = {j for j, e in r.events if e == "shrink"}
    assert shrinks, r.events
    steps = [t for t in seen if t[3] is not None]
    assert len(steps) >= 3
    m = 6
    for j, lam, nnow, before, after in steps:
        if expand == "drop":
            assert np.array_equal(before, after)
            continue
        a, a0 = lam[nnow - 1], lam[0]
        c, e = (a + 10.5) / 2, (10.5 - a) / 2
        p = _cheb_T(m, (d - c) / e) / _cheb_T(m, np.array([(a0 - c) / e]))[0]
        ref = p[:, None] * before
        assert np.allclose(after, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
    # chaining: without a shrink in between, a step starts from the last result
    for (j0, _, _, _, after0), (j1, _, _, before1, _) in zip(steps, steps[1:]):
        if j1 == j0 + 1 and j0 not in shrinks:
            assert np.array_equal(before1, after0)


def test_chebsi_powered_drop_matches_and_expands():
    A = W.anderson_3d(6, seed=2)
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    X0 = W.gaussian_block(A.n, 16, 2)
    kw = dict(tol=1e-11, normA=float(np.abs(ev).max()), degree=8, upper=W.gershgorin_bound(A),
              j_warm=2, r_warm=1e-2, je=4, js=1)
    r = chebsi(A, X0, 8, 11, "fix", expand="powered", **kw)
    assert r.converged and np.allclose(r.lam, ev[:8], rtol=1e-10, atol=1e-12)
    assert any(e == "expand" for _, e in r.events)


# ---------------------------------------------------------------------------
# The 'Random' expansion of Sec. 6.4: the counter-based Gaussian columns
# ---------------------------------------------------------------------------
def test_philox_known_answers(golden_dir):
    from oracle.philox import philox4x32_10
    rows = [l.split()[1:] for l in open(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
            if l.startswith("kat ")]
    assert len(rows) == 3
    for r in rows:
        c0, c1, c2, c3, k0, k1, *want = (int(x, 16) for x in r)
        got = philox4x32_10([c0], [c1], [c2], [c3], k0, k1)
        assert [int(g[0]) for g in got] == want


def test_gaussian_columns_are_standard_normal_and_counter_addressed():
    from scipy import stats
    from oracle.philox import gaussian_columns
    Z = gaussian_columns(20000, 6, seed=12345, e=3)
    # marginal: mean 0, variance 1, normal shape (Kolmogorov-Smirnov)
    assert abs(Z.mean()) < 0.01 and abs(Z.var() - 1.0) < 0.02
    assert stats.kstest(Z.ravel(), "norm").pvalue > 1e-3
    # the sine and cosine halves of one Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(Z[:, 0], Z[:, 1])[0, 1]) < 0.03
    # counter addressing: a sub-block is the block of its own size, and the
    # expansion index and the seed give other draws
    assert np.array_equal(gaussian_columns(300, 4, 12345, 3), Z[:300, :4])
    assert not np.allclose(gaussian_columns(300, 4, 12345, 4), Z[:300, :4])
    assert not np.allclose(gaussian_columns(300, 4, 12346, 3), Z[:300, :4])
    assert np.all(np.isfinite(Z))


def test_expansion_variants_order_as_in_sec_6_4():
    """The appended vectors of Sec. 6.4: on a small Anderson Hamiltonian
    (Chebyshev SI) and on c1 (LOBPCG) every variant converges to the dense
    eigenvalues, and the iteration counts order as the paper reports --
    powered X_drop <= X_drop < Random."""
    A = W.anderson_3d(12, seed=2)
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    X0 = W.gaussian_block(A.n, 32, 2)
    kw = dict(tol=1e-10, normA=float(np.abs(ev).max()), degree=8, upper=W.gershgorin_bound(A), j_warm=2,
              r_warm=1e-2, je=4, js=1, max_iter=400, seed=5)
    its = {}
    for ex in ("drop", "powered", "random"):
        r = chebsi(A, X0, 16, 21, "fix", expand=ex, **kw)
        assert r.converged and np.allclose(r.lam, ev[:16], rtol=1e-10, atol=1e-12)
        its[ex] = r.iters
    assert its["powered"] <= its["drop"] < its["random"], its
    A = W.laplacian_2d(32)
    X0 = W.gaussian_block(A.n, 20, 0)
    normA = W.dirichlet_norm((32, 32))
    drop = lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA)
    rand = lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA, expand="random", seed=5)
    assert drop.converged and rand.converged
    assert np.allclose(rand.lam, drop.lam, rtol=1e-10)
    assert drop.iters < rand.iters
