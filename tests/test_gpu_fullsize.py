"""Parity at the full size of the 3D Dirichlet workload: 128^3 grid
(n = 2,097,152, nnz = 14,581,760), k_max = 128, so S = [X, P, W] is 384
columns wide.  The calls use the launch configuration of the timed solve:
blocks with leading dimension 384 (the solver's S and AS buffers), column
offsets of X, P and W inside them, the tensor-core Gram and update in both
block formats (float64 blocks, seven slices; double-float blocks, six
slices), LOBPCG with the fix strategy in the float64 form.

The oracle computes sampled outputs one by one (rows of A V, U C and of the
residual; entries of U^T V); the whole solve is checked through properties
that hold at any size: residuals by the oracle's SpMM on the host,
orthonormality of the eigenvectors, and the closed-form spectrum.
"""
import numpy as np
import pytest

from oracle import blocks as B
from paper_2409_05572_gb300 import workloads as W
from tc_bounds import DF64_RTOL, gram_bound, update_bound

FMTS = {"f64": "ARITH_F64_TC", "df64": "ARITH_DF64_TC"}

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_05572_gb300 import _lib as L  # noqa: E402

GRID = 128
K_MAX = 128
LDS = 3 * K_MAX   # leading dimension of S = [X, P, W] and AS in the solver


@pytest.fixture(scope="module")
def lap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    A = W.laplacian_3d(GRID)
    assert (A.n, A.nnz) == (2_097_152, 14_581_760)
    yield A
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def sample_rows(n, count, seed):
    """Random rows plus the first and last rows, 128-row chunk edges and the
    rows next to a grid-plane boundary."""
    fixed = [0, 1, 127, 128, 129, GRID * GRID - 1, GRID * GRID, n // 2, n - 129, n - 128, n - 1]
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([fixed, rng.choice(n, count, replace=False)]))


def sample_cols(width, count, seed):
    fixed = [0, 1, 63, 64, 127, 128, width - 1] + ([255, 256] if width > 256 else [])
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[c for c in fixed if c < width], rng.choice(width, count, replace=False)]))


def blk(X64, fmt):
    return L.to_df64(X64) if fmt == "df64" else X64


def df64_rows(Yd, rows, cols):
    """float64 host copy of Yd[rows, :cols] (double-float device block)."""
    return L.from_df64(Yd[torch.as_tensor(rows, device="cuda"), :cols]).cpu().numpy()


# ---------------------------------------------------------------------------
# a7: A W with W at column 2 k_max of S
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", ["f64", "df64"])
def test_spmm_full_size_sampled_rows(lap, fmt):
    A = lap
    n, w = A.n, K_MAX
    S64 = W.gaussian_block_cuda(n, LDS, 21)
    Sd = blk(S64, fmt)
    Yd = blk(W.gaussian_block_cuda(n, LDS, 22), fmt)
    untouched = Yd[:, 2 * K_MAX:].clone()
    rp = torch.as_tensor(A.indptr, device="cuda")
    ci = torch.as_tensor(A.indices, device="cuda")
    val = blk(torch.as_tensor(A.data, device="cuda"), fmt)
    L.eig_spmm(n, rp, ci, val, L.EIG_DF64 if fmt == "df64" else L.EIG_F64, w, Sd[:, 2 * K_MAX:], LDS,
               Yd[:, K_MAX:], LDS)
    torch.cuda.synchronize()
    rows = sample_rows(n, 4000, 1)
    Wh = S64[:, 2 * K_MAX:].cpu().numpy()
    Asub = A.to_scipy()[rows]
    ref = B.spmm(Asub, Wh)
    scale = B.spmm(abs(Asub), np.abs(Wh))
    Ys = Yd[torch.as_tensor(rows, device="cuda"), K_MAX:2 * K_MAX]
    got = (L.from_df64(Ys) if fmt == "df64" else Ys).cpu().numpy()
    rt = 4 * DF64_RTOL if fmt == "df64" else 8 * 2.0 ** -53   # seven products and six sums per row
    assert np.all(np.abs(got - ref) <= rt * scale)
    assert torch.equal(Yd[:, 2 * K_MAX:], untouched)


# ---------------------------------------------------------------------------
# a4 / a5 / a8: Gram on the tensor cores, S^T S (symmetric, 384 x 384) and
# S^T [AP, AW] (384 x 256), columns over a wide range of magnitudes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", ["f64", "df64"])
@pytest.mark.parametrize("sym", [True, False])
def test_gram_tc_full_size_sampled_entries(lap, sym, fmt):
    n = lap.n
    scale = torch.tensor(2.0 ** np.random.default_rng(3).integers(-30, 30, LDS), dtype=torch.float64,
                         device="cuda")
    U64 = W.gaussian_block_cuda(n, LDS, 31) * scale
    Ud = blk(U64, fmt)
    if sym:
        a = b = LDS
        V64, Vd, voff = U64, Ud, 0
    else:
        a, b = LDS, 2 * K_MAX
        V64 = W.gaussian_block_cuda(n, LDS, 32)
        Vd, voff = blk(V64, fmt), K_MAX
    G = torch.full((a, b), float("nan"), dtype=torch.float64, device="cuda")
    L.eig_gram(n, a, b, Ud, LDS, Vd[:, voff:], LDS, getattr(L, FMTS[fmt]), sym, G, b)
    assert L.device_status() == 0
    I = sample_cols(a, 20, 5)
    J = sample_cols(b, 20, 6)
    Uh = U64[:, torch.as_tensor(I, device="cuda")].cpu().numpy()
    Vh = V64[:, torch.as_tensor(J + voff, device="cuda")].cpu().numpy()
    ref = B.gram(Uh, Vh)
    got = G.cpu().numpy()[np.ix_(I, J)]
    bound = gram_bound(Uh, Vh, fmt)
    err = np.abs(got - ref)
    assert np.all(err <= bound), np.max(err / bound)
    Gh = G.cpu().numpy()
    assert np.all(np.isfinite(Gh))
    if sym:
        assert np.array_equal(Gh, Gh.T)


# ---------------------------------------------------------------------------
# a11 / a4: block update on the tensor cores, X <- S C (384 -> 256, beta 0)
# and W <- W - Q C (Q = [X, P], 256 -> 128, beta 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", ["f64", "df64"])
@pytest.mark.parametrize("s,c,beta", [(LDS, 2 * K_MAX, 0.0), (2 * K_MAX, K_MAX, 1.0)])
def test_update_tc_full_size_sampled_rows(lap, s, c, beta, fmt):
    n = lap.n
    U64 = W.gaussian_block_cuda(n, LDS, 41)
    Ud = blk(U64, fmt)
    rng = np.random.default_rng(42)
    Cm = rng.standard_normal((s, c)) * 2.0 ** rng.integers(-20, 20, (s, 1))
    Y64 = W.gaussian_block_cuda(n, LDS, 43)
    Yd = blk(Y64.clone(), fmt)
    yoff = LDS - c           # the output block sits at the right end of its buffer
    before = Yd[:, :yoff].clone()
    L.eig_block_update(n, s, c, Ud, LDS, torch.as_tensor(Cm, device="cuda"), c, Yd[:, yoff:], LDS, beta,
                       getattr(L, FMTS[fmt]))
    assert L.device_status() == 0
    rows = sample_rows(n, 4000, 2)
    rt = torch.as_tensor(rows, device="cuda")
    Uh = U64[rt, :s].cpu().numpy()
    Y0 = Y64[rt, yoff:].cpu().numpy()
    ref = Uh @ Cm + beta * Y0
    got = (L.from_df64(Yd[rt, yoff:]) if fmt == "df64" else Yd[rt, yoff:]).cpu().numpy()
    bound = update_bound(Uh, Cm, beta, Y0, fmt)
    err = np.abs(got - ref)
    assert np.all(err <= bound), np.max(err / bound)
    assert torch.equal(Yd[:, :yoff], before)


# ---------------------------------------------------------------------------
# a1: residual R = AX - X diag(lam) into the W columns, column norms
# ---------------------------------------------------------------------------
def test_residual_full_size(lap):
    n, w = lap.n, K_MAX
    X64 = W.gaussian_block_cuda(n, LDS, 51)
    AX64 = W.gaussian_block_cuda(n, LDS, 52)
    lam = np.random.default_rng(53).uniform(0.0, 0.02, w)
    Xd, AXd = L.to_df64(X64), L.to_df64(AX64)
    Sd = L.to_df64(torch.zeros(n, LDS, dtype=torch.float64, device="cuda"))
    xn = torch.empty(w, dtype=torch.float64, device="cuda")
    rn = torch.empty_like(xn)
    L.eig_residual(n, w, Xd, LDS, AXd, LDS, torch.as_tensor(lam, device="cuda"), None, Sd[:, 2 * K_MAX:], LDS,
                   xn, rn, L.EIG_DF64)
    rows = sample_rows(n, 4000, 3)
    rt = torch.as_tensor(rows, device="cuda")
    Xh, AXh = X64[rt, :w].cpu().numpy(), AX64[rt, :w].cpu().numpy()
    Rref, _, _ = B.residual_test(Xh, AXh, lam, 1.0, 1)
    got = L.from_df64(Sd[rt, 2 * K_MAX:]).cpu().numpy()
    assert np.all(np.abs(got - Rref) <= DF64_RTOL * (np.abs(AXh) + np.abs(Xh * lam)))
    # the norms reduce over all n rows: compare with the full columns
    Xf, AXf = X64[:, :w].cpu().numpy(), AX64[:, :w].cpu().numpy()
    assert np.allclose(xn.cpu().numpy(), np.sum(Xf * Xf, axis=0), rtol=1e-11, atol=0)
    Rf = AXf - Xf * lam
    assert np.allclose(rn.cpu().numpy(), np.sum(Rf * Rf, axis=0), rtol=1e-11, atol=0)


# ---------------------------------------------------------------------------
# the whole solve as timed: 64 eigenpairs of the 128^3 Dirichlet Laplacian
# ---------------------------------------------------------------------------
def dirichlet_lowest(dims, k):
    axes = [4 * np.sin(np.arange(1, min(d, k) + 1) * np.pi / (2 * (d + 1))) ** 2 for d in dims]
    tot = axes[0]
    for ax in axes[1:]:
        tot = np.add.outer(tot, ax).ravel()
    return np.sort(tot)[:k]


def test_full_size_lobpcg_fix_properties(lap):
    """The float64 form as timed (tensor-core products by seven slices)."""
    A = lap
    n, nev, tol = A.n, 64, 1e-8
    normA = W.dirichlet_norm((GRID, GRID, GRID))
    X0 = torch.as_tensor(W.gaussian_block(n, K_MAX, 1), device="cuda")
    rp = torch.as_tensor(A.indptr, device="cuda")
    ci = torch.as_tensor(A.indices, device="cuda")
    va = torch.as_tensor(A.data, device="cuda")
    s = L.Solver((rp, ci, va), nev=nev, k_max=K_MAX, strategy="fix", X0=X0, normA=normA, tol=0.5 * tol,
                 form="f64")
    out = s.solve()
    assert out["status"] == 0
    assert out["n_shrink"] > 0 and out["n_expand"] > 0
    assert L.device_status() == 0
    V = s.V().cpu().numpy()
    s.close()
    lam = out["lam"]
    # residuals by the oracle's SpMM in float64: ||A v - lam v|| / ||A|| <= tol
    R = B.spmm(A, V) - V * lam
    rel = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(V, axis=0))
    assert rel.max() <= tol, rel.max()
    # orthonormal eigenvectors (float64 CholeskyQR2 in the final pass; the
    # host Gram itself rounds length-n dot products)
    assert np.max(np.abs(B.gram(V, V) - np.eye(nev))) <= 1e-12
    # closed-form spectrum: the Ritz values of the converged block are
    # within |dlam| <= ||r||^2 / gap of the exact eigenvalues; the 64 lowest
    # of the 128^3 Dirichlet Laplacian are within 1e-10 relative
    exact = dirichlet_lowest((GRID, GRID, GRID), nev)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - exact) / exact) <= 1e-10
