"""Parity of the CUDA path (through the C ABI) against the FP64 oracle, step by
step and for whole solves.  Sizes span several 64-wide tiles and a ragged
tail; tolerances follow from the arithmetic of each form:

* F64 (native float64): round-off of length-n dot products, 1e-13 relative
  to sum |u_i v_i|.
* DF64 (double-float, about 2^-48 per operation): 1e-12 relative to
  sum |u_i v_i|.
* C32 (float32 inputs, compensated Dot2 sums): 1e-9 relative to
  sum |u_i v_i| of the float32-rounded inputs.
* F32: 2e-5 relative.
"""
import math

import numpy as np
import pytest

from oracle import blocks as B
from oracle.chebsi import chebsi as o_chebsi
from oracle.lobpcg import lobpcg as o_lobpcg
from paper_2409_05572_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_05572_gb300 import _lib as L  # noqa: E402

ARITHS = {"f64": L.ARITH_F64, "df64": L.ARITH_DF64, "f32": L.ARITH_F32, "c32": L.ARITH_C32}
RTOL = {"f64": 1e-13, "df64": 1e-12, "c32": 1e-9, "f32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    yield
    torch.cuda.synchronize()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def to_fmt(x_np, arith):
    """Host float64 array -> device block in the element format of arith."""
    t = dev(x_np)
    if arith in ("f64",):
        return t, L.EIG_F64
    if arith == "df64":
        return L.to_df64(t), L.EIG_DF64
    return t.float(), L.EIG_F32


def from_fmt(t, arith):
    if arith == "df64":
        return L.from_df64(t).cpu().numpy()
    return t.double().cpu().numpy()


def rounded(x_np, arith):
    return x_np.astype(np.float32).astype(np.float64) if arith in ("f32", "c32") else x_np


# ---------------------------------------------------------------------------
# a7: SpMM
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("arith", ["f64", "df64", "f32"])
@pytest.mark.parametrize("w", [1, 3, 8, 20, 64, 69, 130, 133, 300])
def test_spmm_parity(arith, w):
    A = W.anderson_3d(9, seed=2)   # n = 729, 7 nnz/row, random values
    n = A.n
    rng = np.random.default_rng(w)
    V = rng.standard_normal((n, w))
    U = rng.standard_normal((n, w))
    rp, ci = dev(A.indptr, torch.int32), dev(A.indices, torch.int32)
    val, _ = to_fmt(A.data, arith)
    Vd, dt = to_fmt(V, arith)
    Ud, _ = to_fmt(U, arith)
    Yd = torch.empty_like(Vd)
    for (alpha, beta, gamma) in ((1.0, 0.0, 0.0), (0.37, -1.25, 0.5)):
        L.eig_spmm(n, rp, ci, val, dt, w, Vd, w, Yd, w, alpha, beta, Ud if gamma else None, w, gamma)
        torch.cuda.synchronize()
        Ar, Vr, Ur = rounded(A.data, arith), rounded(V, arith), rounded(U, arith)
        Ao = W.CSR(n, A.indptr, A.indices, Ar)
        ref = alpha * B.spmm(Ao, Vr) + beta * Vr + gamma * Ur
        scale = np.abs(alpha) * B.spmm(W.CSR(n, A.indptr, A.indices, np.abs(Ar)), np.abs(Vr)) + \
            abs(beta) * np.abs(Vr) + abs(gamma) * np.abs(Ur)
        got = from_fmt(Yd, arith)
        assert np.all(np.abs(got - ref) <= 4 * RTOL[arith] * scale + 1e-300), (arith, w)


def test_spmm_power_law_rows():
    A = W.graph_laplacian(4000, seed=3)   # rows from 3 to hundreds of nonzeros
    n, w = A.n, 37
    V = np.random.default_rng(1).standard_normal((n, w))
    Yd = torch.empty(n, w, dtype=torch.float64, device="cuda")
    L.eig_spmm(n, dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data), L.EIG_F64, w,
               dev(V), w, Yd, w)
    ref = B.spmm(A, V)
    scale = B.spmm(W.CSR(n, A.indptr, A.indices, np.abs(A.data)), np.abs(V))
    assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 1e-13 * scale)


def test_spmm_empty_rows_and_zero_width():
    n = 50
    indptr = np.zeros(n + 1, dtype=np.int32)
    indptr[26:] = 1
    A = W.CSR(n, indptr, np.array([3], dtype=np.int32), np.array([2.5]))
    V = np.arange(n * 4, dtype=np.float64).reshape(n, 4)
    Yd = torch.full((n, 4), 7.0, dtype=torch.float64, device="cuda")
    L.eig_spmm(n, dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data), L.EIG_F64, 4,
               dev(V), 4, Yd, 4)
    ref = B.spmm(A, V)
    assert np.array_equal(Yd.cpu().numpy(), ref)
    L.eig_spmm(n, dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data), L.EIG_F64, 0,
               dev(V), 4, Yd, 4)


# ---------------------------------------------------------------------------
# a4 / a5 / a8: Gram
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("arith", ["f64", "df64", "c32", "f32"])
@pytest.mark.parametrize("a,b,sym", [(7, 5, False), (64, 64, True), (130, 70, False), (150, 150, True)])
def test_gram_parity(arith, a, b, sym):
    n = 5000 + 17
    rng = np.random.default_rng(a * 1000 + b)
    U = rng.standard_normal((n, a))
    V = U.copy() if sym else rng.standard_normal((n, b))
    Ud, _ = to_fmt(U, arith)
    Vd, _ = to_fmt(V, arith)
    G = torch.empty(a, b + 3, dtype=torch.float64, device="cuda")
    L.eig_gram(n, a, b, Ud, a, Vd, b, ARITHS[arith], sym, G, b + 3)
    got = G[:, :b].cpu().numpy()
    Ur, Vr = rounded(U, arith), rounded(V, arith)
    ref = B.gram(Ur, Vr)
    scale = np.abs(Ur).T @ np.abs(Vr)
    assert np.all(np.abs(got - ref) <= RTOL[arith] * scale), np.max(np.abs(got - ref) / scale)
    if sym:
        assert np.array_equal(got, got.T)


def test_gram_deterministic_and_empty():
    n, a = 20000, 96
    U = np.random.default_rng(3).standard_normal((n, a))
    Ud = L.to_df64(dev(U))
    G1 = torch.empty(a, a, dtype=torch.float64, device="cuda")
    G2 = torch.empty_like(G1)
    L.eig_gram(n, a, a, Ud, a, Ud, a, L.ARITH_DF64, True, G1, a)
    L.eig_gram(n, a, a, Ud, a, Ud, a, L.ARITH_DF64, True, G2, a)
    assert torch.equal(G1, G2)
    G0 = torch.full((3, 3), 5.0, dtype=torch.float64, device="cuda")
    L.eig_gram(0, 3, 3, Ud, a, Ud, a, L.ARITH_DF64, False, G0, 3)
    assert torch.count_nonzero(G0) == 0


# ---------------------------------------------------------------------------
# a4 / a11: block update
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("arith", ["f64", "df64", "f32"])
@pytest.mark.parametrize("s,c,beta", [(5, 3, 0.0), (70, 130, 0.0), (150, 64, -1.0)])
def test_update_parity(arith, s, c, beta):
    n = 3000 + 5
    rng = np.random.default_rng(s + c)
    U = rng.standard_normal((n, s))
    Cm = rng.standard_normal((s, c))
    Y0 = rng.standard_normal((n, c))
    Ud, _ = to_fmt(U, arith)
    Yd, _ = to_fmt(Y0, arith)
    L.eig_block_update(n, s, c, Ud, s, dev(Cm), c, Yd, c, beta, ARITHS[arith])
    got = from_fmt(Yd, arith)
    Ur, Yr = rounded(U, arith), rounded(Y0, arith)
    Cr = rounded(Cm, arith)
    ref = Ur @ Cr + beta * Yr
    scale = np.abs(Ur) @ np.abs(Cr) + abs(beta) * np.abs(Yr)
    tol = {"f64": 1e-13, "df64": 1e-12, "f32": 2e-6}[arith]
    assert np.all(np.abs(got - ref) <= tol * scale + 1e-300)


# ---------------------------------------------------------------------------
# a1 / a2: residual, norms, Jacobi preconditioning
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("arith", ["f64", "df64", "f32"])
def test_residual_parity(arith):
    n, w = 4000 + 3, 45
    rng = np.random.default_rng(7)
    X = rng.standard_normal((n, w))
    AX = rng.standard_normal((n, w))
    lam = rng.uniform(-3, 3, w)
    t = rng.uniform(0.1, 2.0, n)
    Xd, dt = to_fmt(X, arith)
    AXd, _ = to_fmt(AX, arith)
    td, _ = to_fmt(t, arith)
    Rd = torch.empty_like(Xd)
    xn = torch.empty(w, dtype=torch.float64, device="cuda")
    rn = torch.empty_like(xn)
    L.eig_residual(n, w, Xd, w, AXd, w, dev(lam), td, Rd, w, xn, rn, dt)
    Xr, AXr, tr = rounded(X, arith), rounded(AX, arith), rounded(t, arith)
    Rref, _, _ = B.residual_test(Xr, AXr, lam, 1.0, 1)
    tol = {"f64": 1e-13, "df64": 1e-12, "f32": 1e-5}[arith]
    scale = np.abs(AXr) + np.abs(Xr * lam)
    assert np.all(np.abs(from_fmt(Rd, arith) - tr[:, None] * Rref) <= tol * tr[:, None] * scale)
    assert np.allclose(xn.cpu().numpy(), np.sum(Xr * Xr, axis=0), rtol=10 * tol)
    assert np.allclose(rn.cpu().numpy(), np.sum(Rref * Rref, axis=0), rtol=100 * tol)


# ---------------------------------------------------------------------------
# a5: CholeskyQR2 (unique Q with positive R diagonal -> elementwise parity)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("w", [1, 9, 64, 100])
def test_cholqr2_parity(arith, w):
    n = 6000 + 11
    Wm = np.random.default_rng(w).standard_normal((n, w))
    Wd, _ = to_fmt(Wm, arith)
    st = L.eig_cholqr2(n, w, Wd, w, ARITHS[arith])
    assert st == 0
    Q = from_fmt(Wd, arith)
    ref = B.cholqr2(Wm)
    assert np.abs(Q - ref).max() < 1e-11
    assert np.linalg.norm(Q.T @ Q - np.eye(w)) < 1e-12


def test_cholqr2_shifted_path():
    n, w = 3000, 12
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((n, w)))
    V, _ = np.linalg.qr(rng.standard_normal((w, w)))
    Wm = U @ np.diag(np.logspace(0, -11, w)) @ V.T
    Wd = dev(Wm)
    st = L.eig_cholqr2(n, w, Wd, w, L.ARITH_F64)
    assert st == 1
    Q = Wd.cpu().numpy()
    assert np.linalg.norm(Q.T @ Q - np.eye(w)) < 1e-12
    # Q captures the column space of W (directions with singular values near
    # 1e-11 are fixed only to about u / sigma, so spans are not compared)
    assert np.linalg.norm(Wm - Q @ (Q.T @ Wm)) < 1e-13 * np.linalg.norm(Wm)


# ---------------------------------------------------------------------------
# a9: small dense eigensolver
# ---------------------------------------------------------------------------
def _sym(s, seed, kind="random"):
    rng = np.random.default_rng(seed)
    if kind == "random":
        M = rng.standard_normal((s, s))
        return M + M.T
    if kind == "clustered":
        Q, _ = np.linalg.qr(rng.standard_normal((s, s)))
        d = np.repeat(np.arange(1, s // 3 + 2, dtype=float), 3)[:s]
        return Q @ np.diag(d) @ Q.T
    if kind == "diag":
        return np.diag(rng.uniform(-1, 1, s))
    raise ValueError(kind)


@pytest.mark.parametrize("s,kind", [(1, "random"), (2, "random"), (3, "random"), (17, "random"),
                                    (60, "clustered"), (64, "diag"), (200, "random"), (384, "random")])
def test_syev_parity(s, kind):
    A = _sym(s, s, kind)
    lam = torch.empty(s, dtype=torch.float64, device="cuda")
    Z = torch.empty(s, s, dtype=torch.float64, device="cuda")
    L.eig_syev(s, dev(A), s, lam, Z, s)
    lam_h, Z_h = lam.cpu().numpy(), Z.cpu().numpy()
    theta, _ = B.rayleigh_ritz(np.eye(s), A)
    nA = max(np.abs(theta).max(), 1e-300)
    assert np.all(np.diff(lam_h) >= 0)
    assert np.abs(lam_h - theta).max() <= 1e-13 * nA * max(1, math.sqrt(s))
    assert np.linalg.norm(Z_h.T @ Z_h - np.eye(s)) <= 1e-13 * s
    assert np.linalg.norm(A @ Z_h - Z_h * lam_h) <= 1e-13 * nA * s


def projected_like_matrix(seed=0):
    """A Rayleigh-Ritz matrix of the shape a float64 LOBPCG solve of the
    128^3 Dirichlet Laplacian meets after soft locking (s = 233): a diagonal
    block of 69 locked Ritz values equal to the lowest closed-form
    eigenvalues (exact multiplicities 3 and 6), coupled only through a dense
    rotation of the remaining 164 values, which contain near-degenerate
    triples spaced at float32 resolution (3e-7 against ||A|| of 7) and a
    spread up to 7.  Returns A and its exact eigenvalues."""
    rng = np.random.default_rng(seed)
    ax = 4 * np.sin(np.arange(1, 12) * np.pi / 258) ** 2
    lap = np.sort(np.add.outer(np.add.outer(ax, ax), ax).ravel())
    locked = lap[:69]
    mid = list(lap[69:99])
    for c in np.linspace(0.018, 0.03, 12):
        mid += [c, c + 3e-7, c + 7e-7]
    top = list(rng.uniform(0.05, 6.9, 164 - len(mid) - 1)) + [6.93]
    rest = np.array(mid + top)
    Q, _ = np.linalg.qr(rng.standard_normal((rest.size, rest.size)))
    A = np.zeros((233, 233))
    A[:69, :69] = np.diag(locked)
    A[69:, 69:] = (Q * rest) @ Q.T
    A = 0.5 * (A + A.T)
    return A, np.sort(np.concatenate([locked, rest]))


def test_syev_degenerate_and_near_degenerate_clusters():
    """Exactly repeated locked values next to near-degenerate triples: the
    float64 eigensolver keeps every eigenpair to float64 accuracy (the float32
    inverse iteration cannot separate triples spaced at its resolution and
    lost orthogonality on such matrices)."""
    A, exact = projected_like_matrix()
    s = A.shape[0]
    lam = torch.empty(s, dtype=torch.float64, device="cuda")
    Z = torch.empty(s, s, dtype=torch.float64, device="cuda")
    L.eig_syev(s, dev(A), s, lam, Z, s)
    lam_h, Z_h = lam.cpu().numpy(), Z.cpu().numpy()
    nA = np.abs(exact).max()
    assert np.abs(lam_h - exact).max() <= 1e-14 * nA
    assert np.abs(Z_h.T @ Z_h - np.eye(s)).max() <= 1e-12
    assert np.abs(A @ Z_h - Z_h * lam_h).max() <= 1e-13 * nA


# ---------------------------------------------------------------------------
# a10: improved Hetmaniuk-Lehoucq basis selection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s,nnow,nlock", [(30, 10, 0), (30, 10, 3), (96, 40, 0), (200, 90, 7)])
def test_hl_trick_parity(s, nnow, nlock):
    _, Z = np.linalg.eigh(_sym(s, s + nnow))
    q = nnow - nlock
    CP = torch.empty(s, q, dtype=torch.float64, device="cuda")
    L.eig_hl_trick(s, nnow, nlock, dev(Z), s, CP, q)
    got = CP.cpu().numpy()
    _, ref = B.hl_trick(Z, nnow, nlock)
    for j in range(q):
        sg = np.sign(got[:, j] @ ref[:, j])
        assert np.abs(sg * got[:, j] - ref[:, j]).max() < 1e-12


# ---------------------------------------------------------------------------
# invalid arguments are rejected before any launch
# ---------------------------------------------------------------------------
def test_invalid_arguments():
    x = torch.zeros(10, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(L.EigError) as e:
        L.eig_gram(10, 4, 4, x, 3, x, 4, L.ARITH_F64, False, x, 4)   # ldu < a
    assert e.value.code == L.EIG_EINVAL
    with pytest.raises(L.EigError):
        L.eig_hl_trick(10, 8, 0, x, 10, x, 8)                         # s - nnow < nnow - nlock
    with pytest.raises(L.EigError):
        L.eig_syev(-1, x, 1, x, x, 1)
    A = W.laplacian_2d(6)
    with pytest.raises(L.EigError) as e:
        L.Solver(A, nev=4, k_max=8, X0=np.zeros((36, 8)), normA=8.0, nes=8)   # nes >= k_max
    assert e.value.code == L.EIG_EINVAL


# ---------------------------------------------------------------------------
# whole solves against the oracle and the closed forms
# ---------------------------------------------------------------------------
def dirichlet_spectrum(dims):
    axes = [4 * np.sin(np.arange(1, d + 1) * np.pi / (2 * (d + 1))) ** 2 for d in dims]
    tot = axes[0]
    for a in axes[1:]:
        tot = np.add.outer(tot, a).ravel()
    return np.sort(tot)


@pytest.fixture(scope="module")
def c1():
    A = W.laplacian_2d(32)
    return A, W.dirichlet_norm((32, 32)), W.gaussian_block(A.n, 20, 0), dirichlet_spectrum((32, 32))


@pytest.mark.parametrize("form", ["df64", "f64"])
@pytest.mark.parametrize("strategy", ["none", "fix", "slope", "slopek"])
def test_c1_lobpcg_parity(c1, form, strategy):
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy=strategy, X0=X0, normA=normA, tol=1e-10, form=form)
    out = s.solve()
    ref = o_lobpcg(A, X0, 10, 15, strategy, tol=1e-10, normA=normA)
    assert out["status"] == 0
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-10
    assert np.max(np.abs(out["lam"] - ex[:10]) / ex[:10]) <= 1e-10
    assert out["resid"].max() <= 2e-10
    # step-by-step: the residual histories agree while rounding is negligible
    m = min(12, len(ref.history), len(out["history"]))
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
    if strategy != "none":
        assert out["n_shrink"] >= 1 and out["n_expand"] >= 1
    # subspace of complete clusters (10 wanted values close a pair)
    V = s.V().cpu().numpy()
    Qv, _ = np.linalg.qr(V)
    Qo, _ = np.linalg.qr(ref.X)
    assert np.linalg.norm(Qv @ Qv.T - Qo @ Qo.T, 2) < 1e-8
    s.close()


@pytest.mark.parametrize("form", ["df64", "f64"])
def test_c1_lobpcg_cuda_core_gram(c1, form):
    """The double-float and float64 forms with their Gram products and
    updates on the CUDA cores (gram_tc = 0: FP32-pipe double-float, native
    FP64) instead of the tensor cores."""
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10, gram_tc=0, form=form)
    out = s.solve()
    ref = o_lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA)
    assert out["status"] == 0
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-10
    assert out["resid"].max() <= 2e-10
    m = min(12, len(ref.history), len(out["history"]))
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
    s.close()


def test_c1_lobpcg_mixed(c1):
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10, form="mixed")
    out = s.solve()
    ref = o_lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA)
    assert out["status"] == 0 and ref.converged
    assert np.max(np.abs(out["lam"] - ex[:10]) / ex[:10]) <= 1e-8
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-8
    assert out["resid"].max() <= 1e-8
    V = s.V().cpu().numpy()
    Qv, _ = np.linalg.qr(V)
    Qo, _ = np.linalg.qr(ref.X)
    assert np.linalg.norm(Qv @ Qv.T - Qo @ Qo.T, 2) < 1e-6
    s.close()


@pytest.mark.parametrize("form", ["df64", "f64"])
def test_lobpcg_3d_several_tiles_closed_form(form):
    A = W.laplacian_3d(20, 22, 24)   # n = 10560
    ex = dirichlet_spectrum((20, 22, 24))
    normA = W.dirichlet_norm((20, 22, 24))
    X0 = W.gaussian_block(A.n, 40, 1)
    s = L.Solver(A, nev=24, k_max=40, strategy="fix", X0=X0, normA=normA, tol=1e-10, form=form)
    out = s.solve()
    assert out["status"] == 0
    assert np.max(np.abs(out["lam"] - ex[:24]) / ex[:24]) <= 1e-10
    assert out["resid"].max() <= 2e-10
    s.close()


@pytest.mark.parametrize("strategy", ["none", "fix"])
def test_lobpcg_cube_repeated_eigenvalues(strategy):
    """3D Dirichlet cube: eigenvalues of multiplicity 3 and 6 (permutations of
    the grid indices), so the projected matrices have exactly repeated Ritz
    values near convergence and nearly reducible tridiagonal forms."""
    d = 14
    A = W.laplacian_3d(d, d, d)   # n = 2744
    ex = dirichlet_spectrum((d, d, d))
    nev, k = 24, 48
    X0 = W.gaussian_block(A.n, k, 7)
    s = L.Solver(A, nev=nev, k_max=k, strategy=strategy, X0=X0, normA=W.dirichlet_norm((d, d, d)), tol=1e-10)
    out = s.solve()
    assert out["status"] == 0
    assert np.max(np.abs(out["lam"] - ex[:nev]) / ex[:nev]) <= 1e-9
    assert out["resid"].max() <= 2e-10
    s.close()


def test_lobpcg_graph_laplacian_jacobi_deflation():
    A = W.graph_laplacian(3000, seed=3)
    M = A.to_scipy()
    ev = np.linalg.eigvalsh(M.toarray())
    X0 = W.gaussian_block(A.n, 24, 3)
    normA = float(ev[-1])
    s = L.Solver(A, nev=12, k_max=24, strategy="fix", X0=X0, normA=normA, tol=1e-9, precond=1,
                 deflate_ones=1, max_iter=800)
    out = s.solve()
    ref = o_lobpcg(A, X0, 12, 17, "fix", tol=1e-9, normA=normA, precond=1.0 / M.diagonal(),
                   u0=np.ones(A.n) / math.sqrt(A.n), max_iter=800)
    assert out["status"] == 0 and ref.converged
    assert np.max(np.abs(out["lam"] - ev[1:13]) / ev[1:13]) <= 1e-9
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-9
    V = s.V().cpu().numpy()
    assert np.abs(V.sum(axis=0)).max() / math.sqrt(A.n) < 1e-9
    s.close()


def hub_graph_laplacian(n=4000, hubs=(1500, 900, 700, 530), seed=9):
    """A ring plus hub vertices joined to many random vertices: rows longer
    than the SpMM's split threshold (512 nonzeros) next to short ones."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows = list(range(n))
    cols = [(i + 1) % n for i in range(n)]
    vals = list(rng.uniform(0.5, 1.5, n))
    for h, deg in enumerate(hubs):
        nb = rng.choice(np.arange(len(hubs), n), deg, replace=False)
        rows += [h] * deg
        cols += list(nb)
        vals += list(rng.uniform(0.5, 1.5, deg))
    Wm = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    Wm = Wm + Wm.T
    Lm = (sp.diags(np.asarray(Wm.sum(axis=1)).ravel()) - Wm).tocsr()
    Lm.sort_indices()
    return W.CSR(n, Lm.indptr.astype(np.int32), Lm.indices.astype(np.int32), Lm.data.astype(np.float64))


@pytest.mark.parametrize("form", ["f64", "df64", "mixed"])
def test_split_rows_of_power_law_graphs(form):
    """Rows with more than 512 nonzeros go through the split SpMM path (one
    CTA per row, partial rows summed in a fixed order); the whole solve
    matches the dense eigenvalues and the oracle, and runs bitwise the same
    twice."""
    A = hub_graph_laplacian()
    deg = np.diff(A.indptr)
    assert (deg > 512).sum() == 4 and deg.max() > 1000
    M = A.to_scipy()
    ev = np.linalg.eigvalsh(M.toarray())
    X0 = W.gaussian_block(A.n, 24, 4)
    normA = float(ev[-1])
    kw = dict(nev=12, k_max=24, strategy="fix", X0=X0, normA=normA, tol=1e-9, precond=1, deflate_ones=1,
              max_iter=800, form=form)
    s = L.Solver(A, **kw)
    out = s.solve()
    again = s.solve()
    s.close()
    ref = o_lobpcg(A, X0, 12, 17, "fix", tol=1e-9, normA=normA, precond=1.0 / M.diagonal(),
                   u0=np.ones(A.n) / math.sqrt(A.n), max_iter=800)
    assert out["status"] == 0 and ref.converged
    tol = 1e-8 if form == "mixed" else 1e-9
    assert np.max(np.abs(out["lam"] - ev[1:13]) / ev[1:13]) <= tol
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= tol
    assert np.array_equal(out["lam"], again["lam"])


@pytest.mark.parametrize("form", ["df64", "f64", "mixed"])
@pytest.mark.parametrize("strategy", ["none", "fix", "slopek"])
def test_chebsi_anderson_parity(form, strategy):
    A = W.anderson_3d(12, seed=2)    # n = 1728, indefinite
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    X0 = W.gaussian_block(A.n, 32, 2)
    ub = W.gershgorin_bound(A)
    normA = float(np.abs(ev).max())
    kw = dict(j_warm=2, r_warm=1e-2, je=4, js=1, jp=2)
    s = L.Solver(A, nev=16, k_max=32, strategy=strategy, X0=X0, normA=normA, tol=1e-11, algo="chebsi",
                 form=form, cheb_degree=10, cheb_upper=ub, max_iter=400, **kw)
    out = s.solve()
    ref = o_chebsi(A, X0, 16, 21, strategy, tol=1e-11, normA=normA, degree=10, upper=ub, max_iter=400, **kw)
    assert out["status"] == 0 and ref.converged
    tol = 1e-8 if form == "mixed" else 1e-10
    assert np.max(np.abs(out["lam"] - ev[:16]) / np.abs(ev[:16])) <= tol
    assert np.max(np.abs(out["lam"] - ref.lam) / np.abs(ref.lam)) <= tol
    assert out["resid"].max() <= 1e-8
    s.close()


@pytest.fixture(scope="module")
def c3_40():
    """The Anderson workload's solver shape (nev = 128, k_max = 256,
    Chebyshev degree 12, default strategy parameters) on a 40^3 lattice
    (n = 64000) the oracle solves in about a minute."""
    A = W.anderson_3d(40, seed=2)
    X0 = W.gaussian_block(A.n, 256, 2)
    ub, normA = W.gershgorin_bound(A), W.norm_estimate(A)
    ref = o_chebsi(A, X0, 128, 133, "fix", tol=1e-9, normA=normA, degree=12, upper=ub, max_iter=400)
    assert ref.converged
    return A, X0, ub, normA, ref


@pytest.mark.parametrize("form", ["f64", "mixed"])
def test_c3_shape_chebsi_parity(c3_40, form):
    A, X0, ub, normA, ref = c3_40
    s = L.Solver(A, nev=128, k_max=256, strategy="fix", X0=X0, normA=normA, tol=1e-9, algo="chebsi",
                 form=form, cheb_degree=12, cheb_upper=ub, max_iter=400)
    out = s.solve()
    V = s.V().cpu().numpy()
    s.close()
    assert out["status"] == 0
    tol = 1e-8 if form == "mixed" else 1e-10
    assert np.max(np.abs(out["lam"] - ref.lam) / np.abs(ref.lam)) <= tol
    # Eq. conv at 1e-9 bounds ||Av - lam v|| / ||A|| by 2e-9 (|lam| <= ||A||)
    R = B.spmm(A, V) - V * out["lam"]
    rel = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(V, axis=0))
    assert rel.max() <= 2e-9
    assert np.max(np.abs(B.gram(V, V) - np.eye(128))) <= 1e-12
    n_sh = sum(1 for _, e in ref.events if e == "shrink")
    assert n_sh >= 1 and out["n_shrink"] >= 1
    if form == "f64":
        m = min(10, len(ref.history), len(out["history"]))
        assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
        assert abs(out["iters"] - ref.iters) <= 1 and out["n_shrink"] == n_sh


@pytest.mark.parametrize("form", ["f64", "df64"])
def test_row_chunked_tensor_core_products(form):
    """tc_chunk_rows: the slice buffers hold 2048 rows and every Gram and
    update runs over row chunks (the last one ragged); the solve matches the
    unchunked one and the closed form."""
    A = W.laplacian_3d(20, 22, 24)   # n = 10560 = 5 x 2048 + 320
    ex = dirichlet_spectrum((20, 22, 24))
    normA = W.dirichlet_norm((20, 22, 24))
    X0 = W.gaussian_block(A.n, 40, 1)
    kw = dict(nev=24, k_max=40, strategy="fix", X0=X0, normA=normA, tol=1e-10, form=form)
    s = L.Solver(A, tc_chunk_rows=2048, **kw)
    out = s.solve()
    s.close()
    s = L.Solver(A, **kw)
    ref = s.solve()
    s.close()
    assert out["status"] == 0 and ref["status"] == 0
    assert np.max(np.abs(out["lam"] - ex[:24]) / ex[:24]) <= 1e-10
    assert np.max(np.abs(out["lam"] - ref["lam"]) / ref["lam"]) <= 1e-11
    assert out["resid"].max() <= 2e-10


def test_norm_estimated_when_not_given(c1):
    """normA = 0 (None in the binding): eig_create takes the Gershgorin bound
    of ||A||_2 (8 for the 2D Laplacian, against the exact 7.98...), so the
    stopping test is that much stricter and the solve still reaches the
    closed form."""
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, tol=1e-10)
    out = s.solve()
    s.close()
    assert out["status"] == 0
    assert out["normA"] == 8.0 and normA < 8.0
    assert np.max(np.abs(out["lam"] - ex[:10]) / ex[:10]) <= 1e-10


def test_solver_reuse_gives_identical_results(c1):
    A, normA, X0, _ = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10)
    a = s.solve()
    b = s.solve()
    assert np.array_equal(a["lam"], b["lam"]) and a["iters"] == b["iters"]
    s.close()


def test_float32_csr_values_are_widened_exactly(c1):
    """eig_csr.val_dtype = EIG_F32: the 2-D Laplacian's values are exact in
    float32, so host and device float32 CSR give the float64 solve bit for
    bit."""
    A, normA, X0, _ = c1
    ref = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10)
    r = ref.solve()
    ref.close()
    A32 = W.CSR(A.n, A.indptr, A.indices, A.data.astype(np.float32))
    s = L.Solver(A32, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10)
    a = s.solve()
    s.close()
    dv = (torch.as_tensor(A.indptr, device="cuda"), torch.as_tensor(A.indices, device="cuda"),
          torch.as_tensor(A.data.astype(np.float32), device="cuda"))
    d = L.Solver(dv, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10)
    b = d.solve()
    d.close()
    for out in (a, b):
        assert out["status"] == 0 and out["iters"] == r["iters"]
        assert np.array_equal(out["lam"], r["lam"])


@pytest.mark.parametrize("form", ["df64", "f64", "mixed"])
def test_final_pass_is_a_float64_rayleigh_ritz(c1, form):
    """Every form ends with float64 CholeskyQR2 of the converged block and a
    float64 Rayleigh-Ritz on it: the returned vectors are orthonormal and the
    returned values are the Ritz values of A on them, to float64 round-off,
    whatever precision the iteration ran in."""
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10, form=form)
    out = s.solve()
    assert out["status"] == 0
    V = s.V().cpu().numpy()
    s.close()
    assert np.linalg.norm(V.T @ V - np.eye(10), 2) <= 1e-13
    H = V.T @ (A.to_scipy() @ V)
    H = (H + H.T) / 2
    assert np.max(np.abs(np.linalg.eigvalsh(H) - out["lam"])) <= 1e-14 * normA
    assert np.max(np.abs(H - np.diag(out["lam"]))) <= 1e-13 * normA
    R = A.to_scipy() @ V - V * out["lam"]
    want = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(V, axis=0))
    assert np.allclose(want, out["resid"], rtol=1e-6, atol=1e-15)


# ---------------------------------------------------------------------------
# Algorithm 2 (SD) and the powered X_drop expansion of subspace iteration
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("form", ["df64", "f64", "mixed"])
@pytest.mark.parametrize("strategy", ["none", "fix"])
def test_sd_parity(form, strategy):
    from oracle.sd import sd
    A = W.laplacian_2d(16, 12)
    ex = np.sort(np.add.outer(4 * np.sin(np.arange(1, 17) * np.pi / 34) ** 2,
                              4 * np.sin(np.arange(1, 13) * np.pi / 26) ** 2).ravel())
    X0 = W.gaussian_block(A.n, 12, 5)
    kw = dict(j_warm=3, r_warm=1e-3, je=6, js=1, jp=3)
    normA = W.dirichlet_norm((16, 12))
    s = L.Solver(A, nev=6, k_max=12, strategy=strategy, X0=X0, normA=normA, tol=1e-10, algo="sd",
                 form=form, max_iter=3000, nes=8, **kw)
    out = s.solve()
    ref = sd(A, X0, 6, 8, strategy, tol=1e-10, normA=normA, max_iter=3000, **kw)
    assert out["status"] == 0 and ref.converged
    tol = 1e-8 if form == "mixed" else 1e-10
    assert np.max(np.abs(out["lam"] - ex[:6]) / ex[:6]) <= tol
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= tol
    if form != "mixed":
        m = min(10, len(ref.history))
        assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
    if strategy == "fix":
        assert out["n_expand"] >= 1
    s.close()


@pytest.mark.parametrize("form", ["f64", "df64"])
def test_lobpcg_random_expansion_parity(c1, form):
    """The 'Random' variant of Sec. 6.4: the expansion appends counter-based
    Gaussian columns (the same definition on both sides), so the histories
    agree after the expansions too."""
    A, normA, X0, ex = c1
    s = L.Solver(A, nev=10, k_max=20, strategy="fix", X0=X0, normA=normA, tol=1e-10, form=form,
                 expand_random=1, seed=2024)
    out = s.solve()
    s.close()
    ref = o_lobpcg(A, X0, 10, 15, "fix", tol=1e-10, normA=normA, expand="random", seed=2024)
    assert out["status"] == 0 and ref.converged
    assert out["n_expand"] >= 1
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-10
    assert np.max(np.abs(out["lam"] - ex[:10]) / ex[:10]) <= 1e-10
    first_exp = min(j for j, e in ref.events if e == "expand")
    m = min(len(ref.history), len(out["history"]), first_exp + 8)
    assert m > first_exp + 1
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)


def test_chebsi_random_expansion_parity():
    A = W.anderson_3d(12, seed=2)
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    X0 = W.gaussian_block(A.n, 32, 2)
    ub = W.gershgorin_bound(A)
    normA = float(np.abs(ev).max())
    kw = dict(j_warm=2, r_warm=1e-2, je=4, js=1)
    s = L.Solver(A, nev=16, k_max=32, strategy="fix", X0=X0, normA=normA, tol=1e-11, algo="chebsi",
                 cheb_degree=10, cheb_upper=ub, max_iter=400, expand_random=1, seed=77, **kw)
    out = s.solve()
    s.close()
    ref = o_chebsi(A, X0, 16, 21, "fix", tol=1e-11, normA=normA, degree=10, upper=ub, max_iter=400,
                   expand="random", seed=77, **kw)
    assert out["status"] == 0 and ref.converged and out["n_expand"] >= 1
    assert np.max(np.abs(out["lam"] - ev[:16]) / np.abs(ev[:16])) <= 1e-10
    first_exp = min(j for j, e in ref.events if e == "expand")
    m = min(len(ref.history), len(out["history"]), first_exp + 6)
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)


@pytest.mark.parametrize("strategy", ["fix", "slopek"])
def test_lobpcg_aggressive_warmup_parity(c1, strategy):
    """The first-pair warm-up gate of the paper's closing remarks
    (warm_first, r_warm = 1e-1): same decisions and results as the oracle's
    strategy with the same gate, and the first shrink comes earlier than with
    the default gate."""
    A, normA, X0, ex = c1
    kw = dict(warm_first=1, r_warm=1e-1)
    s = L.Solver(A, nev=10, k_max=20, strategy=strategy, X0=X0, normA=normA, tol=1e-10, **kw)
    out = s.solve()
    s.close()
    ref = o_lobpcg(A, X0, 10, 15, strategy, tol=1e-10, normA=normA, warm_first=True, r_warm=1e-1)
    base = o_lobpcg(A, X0, 10, 15, strategy, tol=1e-10, normA=normA)
    assert out["status"] == 0 and ref.converged
    assert np.max(np.abs(out["lam"] - ref.lam) / ref.lam) <= 1e-10
    assert np.max(np.abs(out["lam"] - ex[:10]) / ex[:10]) <= 1e-10
    m = min(12, len(ref.history), len(out["history"]))
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
    # the active widths are the oracle's while the histories agree
    mw = min(m, len(ref.widths), len(out["widths"]))
    assert list(out["widths"][:mw]) == list(ref.widths[:mw])
    first = min(j for j, e in ref.events if e == "shrink")
    first_base = min(j for j, e in base.events if e == "shrink")
    assert first < first_base


def test_chebsi_powered_drop_parity():
    A = W.anderson_3d(12, seed=2)
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    X0 = W.gaussian_block(A.n, 32, 2)
    ub = W.gershgorin_bound(A)
    normA = float(np.abs(ev).max())
    kw = dict(j_warm=2, r_warm=1e-2, je=4, js=1)
    s = L.Solver(A, nev=16, k_max=32, strategy="fix", X0=X0, normA=normA, tol=1e-11, algo="chebsi",
                 cheb_degree=10, cheb_upper=ub, max_iter=400, expand_powered=1, **kw)
    out = s.solve()
    ref = o_chebsi(A, X0, 16, 21, "fix", tol=1e-11, normA=normA, degree=10, upper=ub, max_iter=400,
                   expand="powered", **kw)
    assert out["status"] == 0 and ref.converged
    assert np.max(np.abs(out["lam"] - ev[:16]) / np.abs(ev[:16])) <= 1e-10
    assert np.max(np.abs(out["lam"] - ref.lam) / np.abs(ref.lam)) <= 1e-10
    m = min(8, len(ref.history))
    assert np.allclose(out["history"][:m], ref.history[:m], rtol=1e-6)
    s.close()
