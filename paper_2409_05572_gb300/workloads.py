"""Seeded synthetic inputs for the shrink-and-expand block eigensolvers.

This module builds the matrices, initial blocks and request streams that both
the CUDA path and the FP64 oracle consume.  It holds none of the eigensolver's
arithmetic: it only assembles CSR matrices, draws seeded random numbers and
states closed-form matrix norms that are passed in as inputs.

Random numbers come from NumPy's Philox4x32-10 counter-based generator
(Salmon et al., SC'11): the same seed gives the same stream on x86 and Arm.

Workloads (stand-ins for the SuiteSparse matrices of the paper's Table 1,
which are not reconstructed here):

* ``laplacian_2d`` / ``laplacian_3d``: Dirichlet 5-/7-point finite-difference
  Laplacians on a regular grid (PDE-stencil class).
* ``anderson_3d``: periodic 7-point hopping Hamiltonian with i.i.d. uniform
  on-site disorder (disordered-Hamiltonian class).
* ``graph_laplacian``: L = D - W of a Chung-Lu power-law random graph made
  connected by a random Hamiltonian cycle (graph class).
* ``serving_stream``: Poisson arrivals of grid Laplacians plus a random
  positive diagonal.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Square CSR matrix with int32 indices and float64 values (row-major)."""

    n: int
    indptr: np.ndarray   # int32[n+1]
    indices: np.ndarray  # int32[nnz]
    data: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    # Philox key = seed; disjoint streams via the top word of the 256-bit counter.
    return np.random.Generator(np.random.Philox(key=seed, counter=[0, 0, 0, stream]))


def _from_coo(n, rows, cols, vals) -> CSR:
    import scipy.sparse as sp
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64))


def _grid_stencil(dims, periodic: bool, diag: np.ndarray, hop: float) -> CSR:
    """Nearest-neighbour stencil on a grid of shape ``dims`` (x fastest)."""
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    rows = [idx]
    cols = [idx]
    vals = [diag.astype(np.float64)]
    stride = 1
    for ax, d in enumerate(dims):
        c = coords[ax]
        for step in (-1, 1):
            nb = c + step
            if periodic:
                nb_w = nb % d
                ok = np.ones(n, dtype=bool)
            else:
                nb_w = nb
                ok = (nb >= 0) & (nb < d)
            j = idx + (nb_w - c) * stride
            rows.append(idx[ok])
            cols.append(j[ok])
            vals.append(np.full(int(ok.sum()), hop))
        stride *= d
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    """Dirichlet 5-point Laplacian (diagonal 4, off-diagonal -1)."""
    ny = nx if ny is None else ny
    return _grid_stencil((nx, ny), False, np.full(nx * ny, 4.0), -1.0)


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """Dirichlet 7-point Laplacian (diagonal 6, off-diagonal -1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _grid_stencil((nx, ny, nz), False, np.full(nx * ny * nz, 6.0), -1.0)


def dirichlet_norm(dims) -> float:
    """Largest eigenvalue of the Dirichlet grid Laplacian: sum over axes of
    4 sin^2(N pi / (2(N+1))).  Used as the matrix 2-norm input of Eq. conv."""
    return float(sum(4.0 * math.sin(d * math.pi / (2 * (d + 1))) ** 2 for d in dims))


def anderson_3d(L: int, disorder: float = 16.5, seed: int = 2) -> CSR:
    """Periodic L^3 Anderson Hamiltonian: hopping -1 to the 6 neighbours and
    on-site energies i.i.d. uniform on [-disorder/2, disorder/2]."""
    n = L ** 3
    eps = _rng(seed).uniform(-disorder / 2, disorder / 2, size=n)
    return _grid_stencil((L, L, L), True, eps, -1.0)


def shifted_grid(dims, diag_shift: np.ndarray) -> CSR:
    """Dirichlet grid Laplacian plus a diagonal (serving requests)."""
    base = 2.0 * len(dims)
    return _grid_stencil(tuple(dims), False, base + diag_shift, -1.0)


def graph_laplacian(n: int, alpha: float = 2.5, mean_degree: float = 10.0,
                    seed: int = 3) -> CSR:
    """Weighted Laplacian L = D - W of a connected power-law random graph.

    Expected degrees w_i proportional to (i+1)^(-1/(alpha-1)), capped at
    sqrt(sum w) and scaled so that, with the random Hamiltonian cycle that
    makes the graph connected (2 per vertex), the mean degree is
    ``mean_degree``.  Edge endpoints are drawn independently with
    probability proportional to w (edge-sampling form of the Chung-Lu model);
    self loops are dropped and repeated edges merged by summing weights.
    Every edge weight is uniform on [0.5, 1.5].
    """
    rng = _rng(seed)
    target = mean_degree - 2.0
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (alpha - 1.0))
    w *= target / w.mean()
    cap = math.sqrt(w.sum())
    w = np.minimum(w, cap)
    w *= target / w.mean()
    m = int(round(n * target / 2))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    v = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    keep = u != v
    u, v = u[keep], v[keep]
    wt = rng.uniform(0.5, 1.5, size=u.size)
    perm = rng.permutation(n).astype(np.int64)
    cu, cv = perm, np.roll(perm, -1)
    cw = rng.uniform(0.5, 1.5, size=n)
    eu = np.concatenate([u, cu])
    ev = np.concatenate([v, cv])
    ew = np.concatenate([wt, cw])
    rows = np.concatenate([eu, ev])
    cols = np.concatenate([ev, eu])
    vals = -np.concatenate([ew, ew])
    deg = np.zeros(n)
    np.add.at(deg, rows, -vals)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, deg])
    return _from_coo(n, rows, cols, vals)


def gershgorin_bound(A: CSR) -> float:
    """max_i sum_j |a_ij|, an upper bound on the 2-norm of A."""
    absrow = np.add.reduceat(np.abs(A.data), A.indptr[:-1].astype(np.int64))
    empty = np.diff(A.indptr) == 0
    absrow[empty] = 0.0
    return float(absrow.max())


def norm_estimate(A: CSR, steps: int = 60, seed: int = 11) -> float:
    """Largest |Ritz value| of a fixed-seed ``steps``-step Lanczos run with full
    reorthogonalisation: a lower bound on ||A||_2 used as the matrix norm
    input of Eq. conv when no closed form is known."""
    M = A.to_scipy()
    q = _rng(seed).standard_normal(A.n)
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    b = 0.0
    qprev = np.zeros_like(q)
    for _ in range(min(steps, A.n)):
        z = M @ q - b * qprev
        a = float(q @ z)
        z -= a * q
        for qq in Q:
            z -= (qq @ z) * qq
        b = float(np.linalg.norm(z))
        alpha.append(a)
        beta.append(b)
        if b < 1e-14:
            break
        qprev, q = q, z / b
        Q.append(q)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    return float(np.max(np.abs(np.linalg.eigvalsh(T))))


def gaussian_block(n: int, k: int, seed: int) -> np.ndarray:
    """n x k row-major block of i.i.d. standard normals (Philox, key=seed)."""
    return _rng(seed).standard_normal((n, k))


def gaussian_block_cuda(n: int, k: int, seed: int):
    """n x k row-major float64 block of i.i.d. standard normals drawn on the
    current CUDA device by PyTorch's seeded Philox generator: test inputs of
    full size (gigabytes), which NumPy would take tens of seconds to draw.
    Whatever the oracle needs of it is copied to the host."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn(n, k, dtype=torch.float64, device="cuda", generator=g)


@dataclass
class Request:
    rid: int
    arrival_s: float
    dims: tuple
    diag_shift: np.ndarray
    nev: int
    k_max: int
    seed: int

    def matrix(self) -> CSR:
        return shifted_grid(self.dims, self.diag_shift)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))


def serving_stream(count: int = 2000, rate: float = 200.0, seed: int = 4,
                   n_lo: float = 1e4, n_hi: float = 1e6,
                   nev_lo: int = 8, nev_hi: int = 128) -> list[Request]:
    """Poisson request stream: 2D or 3D Dirichlet Laplacian (fair coin) with
    n log-uniform on [n_lo, n_hi] (grid side round(n^(1/d))), plus a diagonal
    uniform on [0, 1]; nev uniform on {nev_lo..nev_hi}; k_max = 2 nev."""
    g = _rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(count):
        rr = _rng(seed, stream=r + 1)
        d = 2 if rr.random() < 0.5 else 3
        n = math.exp(rr.uniform(math.log(n_lo), math.log(n_hi)))
        side = max(2, int(round(n ** (1.0 / d))))
        dims = (side,) * d
        nev = int(rr.integers(nev_lo, nev_hi + 1))
        shift = rr.uniform(0.0, 1.0, size=side ** d)
        out.append(Request(r, float(t[r]), dims, shift, nev, 2 * nev, seed * 100003 + r))
    return out
