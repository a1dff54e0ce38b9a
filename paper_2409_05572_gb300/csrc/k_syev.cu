// Small dense symmetric eigensolver of the Rayleigh-Ritz step (arXiv:2409.05572,
// Algorithms 1 and 3: "compute the spectral decomposition A_p = Z Lambda Z^H").
//
// GB300 executes scalar FP64 with very long latency (a Givens rotation of the
// sequential QL chain costs about 1 us in float64), so the eigensolver is
// split in two stages:
//
//  1. float32 decomposition: Householder tridiagonalisation (cooperative,
//     grid-synchronised kernel, one warp per row of the trailing matrix),
//     eigenvalues of the tridiagonal by bisection and eigenvectors by inverse
//     iteration with Gram-Schmidt inside clusters (all parallel; the
//     sequential implicit QL with Wilkinson shifts of Bowdler, Martin, Reinsch
//     and Wilkinson 1968 with row-parallel accumulation of its rotations is
//     kept behind EIG_TRIDIAG=ql), and a warp-per-vector back-transformation.
//  2. refinement to float64 accuracy with the iteration of Ogita and Aishima
//     (Japan J. Indust. Appl. Math. 35, 2018): with R = I - X^T X and
//     S = X^T A X, lambda_i = S_ii / (1 - R_ii) and X <- X (I + E),
//     E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) for separated
//     pairs, E_ij = R_ij / 2 inside clusters of nearly equal eigenvalues.  The
//     products run in this library's double-float Gram / update kernels (all
//     SMs, no sequential chain).  Clusters are finally diagonalised by a
//     cyclic Jacobi iteration on their (small) block of X^T A X.
//
// The float64 QL path (stage 1 in float64, no refinement) is kept as
// syev_qr64 for comparison and testing.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "blocks.cuh"
#include "small.cuh"

namespace cg = cooperative_groups;

namespace eig {

template <typename R> struct RealT;
template <> struct RealT<float> {
  static __device__ __forceinline__ float eps() { return 1.1920928955078125e-07f; }
  static __device__ __forceinline__ float tiny() { return 1.1754944e-38f; }
  // inverse-iteration clusters: consecutive eigenvalues closer than this
  // fraction of ||T||_1 are orthogonalised together
  static __device__ __forceinline__ float ortol() { return 1e-5f; }
  static __device__ __forceinline__ float big() { return 1e20f; }
  static __device__ __forceinline__ float hyp(float a, float b) { return hypotf(a, b); }
  static constexpr float lo = 1e-35f, hi = 1e35f;
};
template <> struct RealT<double> {
  static __device__ __forceinline__ double eps() { return 2.220446049250313e-16; }
  static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }
  static __device__ __forceinline__ double ortol() { return 1e-9; }
  static __device__ __forceinline__ double big() { return 1e150; }
  static __device__ __forceinline__ double hyp(double a, double b) { return hypot(a, b); }
  static constexpr double lo = 1e-280, hi = 1e280;
};

template <typename R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  // 256-thread block reduction; all threads get the result
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R t = 0;
  for (int i = 0; i < 8; ++i) t += red[i];
  return t;
}

// ---------------------------------------------------------------------------
// stage 1 kernels (templated on the working precision R)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void copy_sym_kernel(int s, const double* __restrict__ A, int64_t lda, R* __restrict__ Wm) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(s) * s) return;
  const int i = int(idx / s), j = int(idx % s);
  Wm[idx] = R(0.5 * (A[int64_t(i) * lda + j] + A[int64_t(j) * lda + i]));
}

// Householder tridiagonalisation T = Q^T A Q, Q = H_0 ... H_{s-3},
// H_k = I - tau_k v_k v_k^T (v_k in row k of Vh, entries k+1..s-1).
template <typename R>
__global__ void __launch_bounds__(256) sytrd_kernel(int s, R* __restrict__ Wm, R* __restrict__ Vh,
                                                    R* __restrict__ tau, R* __restrict__ d, R* __restrict__ e,
                                                    R* __restrict__ p) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ unsigned char shraw[];
  R* vsh = reinterpret_cast<R*>(shraw);
  R* psh = vsh + s;
  __shared__ R red[8];
  const int nb = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int gw = b * 8 + warp, nw = nb * 8;
  for (int k = 0; k + 2 < s; ++k) {
    const int m = s - k - 1;  // x = A[k+1:, k] = A[k, k+1:] (symmetric storage)
    const R* rowk = Wm + int64_t(k) * s + (k + 1);
    R part = 0, part_tail = 0;
    for (int i = t; i < m; i += blockDim.x) {
      const R x = rowk[i];
      vsh[i] = x;
      part += x * x;
      if (i > 0) part_tail += x * x;
    }
    const R nrm2 = block_sum(part, red);
    const R tail2 = block_sum(part_tail, red);
    const R x0 = vsh[0];
    R tk, alpha;
    if (tail2 == R(0)) {
      tk = 0;
      alpha = x0;
    } else {
      const R nrm = sqrt(nrm2);
      alpha = x0 >= R(0) ? -nrm : nrm;
      const R v0 = x0 - alpha;
      tk = R(2) / (tail2 + v0 * v0);
      __syncthreads();
      if (t == 0) vsh[0] = v0;
    }
    __syncthreads();
    if (b == 0) {
      for (int i = t; i < m; i += blockDim.x) Vh[int64_t(k) * s + k + 1 + i] = vsh[i];
      if (t == 0) {
        tau[k] = tk;
        e[k] = alpha;
        d[k] = Wm[int64_t(k) * s + k];
      }
    }
    if (tk != R(0)) {
      for (int i = gw; i < m; i += nw) {
        const R* wr = Wm + int64_t(k + 1 + i) * s + (k + 1);
        R acc = 0;
        for (int j = lane; j < m; j += 32) acc += wr[j] * vsh[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) p[i] = tk * acc;
      }
    }
    grid.sync();
    if (tk != R(0)) {
      R pv = 0;
      for (int i = t; i < m; i += blockDim.x) {
        const R pi = p[i];
        psh[i] = pi;
        pv += pi * vsh[i];
      }
      const R K = R(0.5) * tk * block_sum(pv, red);
      for (int i = gw; i < m; i += nw) {
        const R vi = vsh[i];
        const R wi = psh[i] - K * vi;
        R* wr = Wm + int64_t(k + 1 + i) * s + (k + 1);
        for (int j = lane; j < m; j += 32) wr[j] -= vi * (psh[j] - K * vsh[j]) + wi * vsh[j];
      }
    }
    grid.sync();
  }
  if (b == 0 && t == 0) {
    if (s >= 2) {
      d[s - 2] = Wm[int64_t(s - 2) * s + (s - 2)];
      e[s - 2] = Wm[int64_t(s - 1) * s + (s - 2)];
    }
    d[s - 1] = Wm[int64_t(s - 1) * s + (s - 1)];
    e[s - 1] = 0;
  }
}

template <typename R>
__global__ void small_tridiag_kernel(int s, const R* Wm, R* d, R* e, R* tau) {
  if (threadIdx.x != 0) return;
  d[0] = Wm[0];
  e[0] = 0;
  tau[0] = 0;
  if (s == 2) {
    d[1] = Wm[3];
    e[0] = Wm[2];
    e[1] = 0;
    tau[1] = 0;
  }
}

// Implicit QL with Wilkinson shifts on (d, e), e[i] = T[i+1][i], one thread,
// d and e in shared memory.  Every Givens rotation applied to eigenvector
// columns (i, i+1) is appended: z_i <- c z_i - s z_{i+1},
// z_{i+1} <- s z_i + c z_{i+1}.
template <typename R>
__global__ void tql_kernel(int s, R* __restrict__ dg, R* __restrict__ eg, int* __restrict__ ri, R* __restrict__ rc,
                           R* __restrict__ rs, int64_t cap, int64_t* nrot, int* status) {
  extern __shared__ unsigned char shraw[];
  R* d = reinterpret_cast<R*>(shraw);
  R* e = d + s;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    d[i] = dg[i];
    e[i] = eg[i];
  }
  __syncthreads();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const R eps = RealT<R>::eps();
  int64_t cnt = 0;
  int st = 0;
  e[s - 1] = 0;
  for (int l = 0; l < s && st == 0; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m < s - 1; ++m) {
        const R dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) {
        st = 1;
        break;
      }
      R g = (d[l + 1] - d[l]) / (R(2) * e[l]);
      R r = RealT<R>::hyp(g, R(1));
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      R sn = 1, cs = 1, p = 0;
      bool early = false;
      for (int i = m - 1; i >= l; --i) {
        const R f = sn * e[i];
        const R bb = cs * e[i];
        // correctly rounded square root and divisions keep c^2 + s^2 = 1 to
        // one ulp; an approximate reciprocal square root biases every
        // rotation and the eigenvectors lose orthogonality over the chain
        const R hh = f * f + g * g;
        if (hh > RealT<R>::lo && hh < RealT<R>::hi)
          r = sqrt(hh);
        else
          r = RealT<R>::hyp(f, g);
        e[i + 1] = r;
        if (r == R(0)) {
          d[i + 1] -= p;
          e[m] = 0;
          early = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * sn + R(2) * cs * bb;
        p = sn * r;
        d[i + 1] = g + p;
        g = cs * r - bb;
        if (cnt < cap) {
          ri[cnt] = i;
          rc[cnt] = cs;
          rs[cnt] = sn;
        }
        ++cnt;
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0;
    }
  }
  if (cnt > cap) st = 2;
  *nrot = cnt < cap ? cnt : cap;
  *status = st;
  for (int i = 0; i < s; ++i) {
    dg[i] = d[i];
    eg[i] = e[i];
  }
}

// ---------------------------------------------------------------------------
// Parallel tridiagonal eigenvectors (float32 stage, default): eigenvalues by
// bisection on Sturm counts (one thread per eigenvalue), eigenvectors by
// inverse iteration with the pivoted LU of T - sigma_j I (one thread per
// vector; after LAPACK's stebz / stein), two passes, each followed by
// classical Gram-Schmidt with re-orthogonalisation inside clusters of
// eigenvalues closer than 1e-5 ||T||_1 (one CTA per cluster).
// No step is a sequential chain over all eigenvalues.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int sturm_count(int s, const R* d, const R* e2, R x, R pivmin) {
  int cnt = 0;
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < R(0);
  for (int k = 1; k < s; ++k) {
    q = (d[k] - x) - e2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < R(0);
  }
  return cnt;
}

// lam[i] = i-th smallest eigenvalue of T (d, e; e[k] = T[k+1][k]) by
// multisection on Sturm counts: one warp per eigenvalue, the 32 lanes count
// at 32 interior points of the current interval, which shrinks to the
// sub-interval holding eigenvalue i (33 times shorter per round), until its
// width is eps ||T|| (eps of the working precision R)
template <typename R>
__global__ void __launch_bounds__(128) bisect_kernel(int s, const R* __restrict__ dg, const R* __restrict__ eg,
                                                     R* __restrict__ lam) {
  extern __shared__ unsigned char shb[];
  R* d = reinterpret_cast<R*>(shb);
  R* e2 = d + s;
  __shared__ R bounds[4];
  const R eps = RealT<R>::eps();
  for (int k = threadIdx.x; k < s; k += blockDim.x) {
    d[k] = dg[k];
    e2[k] = k + 1 < s ? eg[k] * eg[k] : R(0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R gl = d[0], gu = d[0], emax = 0;
    for (int k = 0; k < s; ++k) {
      const R r = (k > 0 ? fabs(eg[k - 1]) : R(0)) + (k + 1 < s ? fabs(eg[k]) : R(0));
      gl = fmin(gl, d[k] - r);
      gu = fmax(gu, d[k] + r);
      emax = fmax(emax, e2[k]);
    }
    const R pivmin = RealT<R>::tiny() * fmax(R(1), emax);
    const R tn = fmax(fabs(gl), fabs(gu));
    bounds[0] = gl - R(2) * eps * tn - R(2) * pivmin;
    bounds[1] = gu + R(2) * eps * tn + R(2) * pivmin;
    bounds[2] = pivmin;
    bounds[3] = eps * tn;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= s) return;  // whole warps leave together
  R lo = bounds[0], hi = bounds[1];
  const R pivmin = bounds[2], atol = bounds[3];
  for (int round = 0; round < 40; ++round) {
    if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + atol) break;
    const R step = (hi - lo) / R(33);
    const R x = lo + step * R(lane + 1);
    const bool above = x < hi && sturm_count<R>(s, d, e2, x, pivmin) > i;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    // lanes 0 .. f-1 count at most i (eigenvalue i lies above their points)
    const int f = m ? __ffs(m) - 1 : 32;
    const R nlo = f > 0 ? __shfl_sync(0xffffffffu, x, f - 1) : lo;
    const R nhi = f < 32 ? __shfl_sync(0xffffffffu, x, f < 32 ? f : 0) : hi;
    if (!(nhi - nlo < hi - lo)) break;  // no progress at this resolution
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) lam[i] = R(0.5) * (lo + hi);
}

// Shifts equal to the eigenvalues: every vector starts from its own
// pseudo-random vector, so the vectors of a repeated eigenvalue stay
// independent without the shift separation of stein (which, at about
// 10 eps ||T|| per member, would push the shifts of a large group of equal
// eigenvalues toward the next distinct one).  Cluster starts: gap to the
// previous eigenvalue at most ortol ||T||_1.  An inverse-iteration vector
// errs by about eps ||T|| / gap in the direction of a neighbour at distance
// gap: pairs closer than ortol ||T|| (1e-9 in float64, 1e-5 in float32) are
// orthogonalised together, and the Ogita-Aishima refinement that follows
// removes the coupling of the farther pairs.  Zero-pivot replacement
// eps ||T||_1.
//
// Float32 cannot resolve eigenvalues whose gaps approach eps32 ||T||: when
// three of them sit within that resolution, inverse iteration from every
// start converges to the same one or two directions, and the Gram-Schmidt
// remainder of the last vector is dominated by neighbouring eigenvectors
// outside the cluster.  The float64 working precision resolves the same
// groups with nine orders of magnitude to spare.
template <typename R>
__global__ void invit_prep_kernel(int s, const R* __restrict__ d, const R* __restrict__ e,
                                  const R* __restrict__ lam, R* __restrict__ sig, int* __restrict__ cstart,
                                  R* __restrict__ pert) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  R nrm = 0;
  for (int k = 0; k < s; ++k)
    nrm = fmax(nrm, fabs(d[k]) + (k > 0 ? fabs(e[k - 1]) : R(0)) + (k + 1 < s ? fabs(e[k]) : R(0)));
  const R ortol = RealT<R>::ortol() * nrm;
  sig[0] = lam[0];
  cstart[0] = 0;
  for (int j = 1; j < s; ++j) {
    sig[j] = lam[j];
    cstart[j] = (lam[j] - lam[j - 1] <= ortol) ? cstart[j - 1] : j;
  }
  *pert = fmax(RealT<R>::eps() * nrm, RealT<R>::tiny());
}

// One inverse-iteration solve per thread j: (T - sig_j I) x = b, b a fixed
// pseudo-random vector (pass 0, which also factors) or column j of ZT (later
// passes); x normalised into column j of ZT (ZT[j s + i]).  Factor arrays are
// [k][j] so that the threads of a warp touch consecutive words.
template <typename R>
__global__ void __launch_bounds__(128) invit_kernel(int s, const R* __restrict__ d, const R* __restrict__ e,
                                                    const R* __restrict__ sig, const R* __restrict__ pertp,
                                                    R* __restrict__ dl, R* __restrict__ dg, R* __restrict__ du,
                                                    R* __restrict__ du2, unsigned char* __restrict__ piv,
                                                    R* __restrict__ b, R* __restrict__ ZT, int pass) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  const int64_t S = s;
  const R pert = *pertp;
  const R big = RealT<R>::big();
#define AT(a, k) a[int64_t(k) * S + j]
  if (pass == 0) {
    const R sg = sig[j];
    for (int k = 0; k < s; ++k) {
      AT(dg, k) = d[k] - sg;
      if (k + 1 < s) {
        AT(dl, k) = e[k];
        AT(du, k) = e[k];
      }
    }
    for (int k = 0; k + 1 < s; ++k) {
      const R a = AT(dg, k), l = AT(dl, k);
      if (fabs(a) >= fabs(l)) {  // no interchange
        const R a2 = a != R(0) ? a : pert;
        const R f = l / a2;
        AT(dl, k) = f;
        AT(dg, k) = a2;
        AT(dg, k + 1) -= f * AT(du, k);
        if (k + 2 < s) AT(du2, k) = R(0);
        AT(piv, k) = 0;
      } else {  // interchange rows k and k + 1
        const R f = a / l;
        const R dk1 = AT(dg, k + 1);
        AT(dg, k) = l;
        AT(dl, k) = f;
        const R t = AT(du, k);
        AT(du, k) = dk1;
        AT(dg, k + 1) = t - f * dk1;
        if (k + 2 < s) {
          const R u1 = AT(du, k + 1);
          AT(du2, k) = u1;
          AT(du, k + 1) = -f * u1;
        }
        AT(piv, k) = 1;
      }
    }
    for (int k = 0; k < s; ++k) {
      const R a = AT(dg, k);
      if (fabs(a) < pert) AT(dg, k) = a < R(0) ? -pert : pert;
    }
    // fixed pseudo-random start (integer hash of (k, j)), entries in [-1, 1)
    for (int k = 0; k < s; ++k) {
      uint32_t h = uint32_t(k) * 0x9E3779B1u ^ (uint32_t(j) * 0x85EBCA77u + 0x27d4eb2fu);
      h ^= h >> 15;
      h *= 0x2C1B3C6Du;
      h ^= h >> 12;
      h *= 0x297A2D39u;
      h ^= h >> 15;
      AT(b, k) = R(int32_t(h)) * R(4.656612873e-10);
    }
  } else {
    R mx = 0;
    for (int k = 0; k < s; ++k) mx = fmax(mx, fabs(ZT[int64_t(j) * S + k]));
    const R sc = mx > R(0) ? R(1) / mx : R(1);
    for (int k = 0; k < s; ++k) AT(b, k) = ZT[int64_t(j) * S + k] * sc;
  }
  // forward: L with the interchanges
  for (int k = 0; k + 1 < s; ++k) {
    if (AT(piv, k) == 0) {
      AT(b, k + 1) -= AT(dl, k) * AT(b, k);
    } else {
      const R t = AT(b, k);
      const R bk1 = AT(b, k + 1);
      AT(b, k) = bk1;
      AT(b, k + 1) = t - AT(dl, k) * bk1;
    }
  }
  // backward: U with two superdiagonals.  A nearly reducible T (repeated
  // eigenvalues) has several tiny pivots, each multiplying the solution by up
  // to ||T|| / pert; the whole vector (solved part and remaining right-hand
  // side alike, x = U^{-1} b being linear) is rescaled before it can overflow.
  R x2 = 0, x1 = 0, nrm = 0;
  for (int k = s - 1; k >= 0; --k) {
    R v = AT(b, k);
    if (k + 1 < s) v -= AT(du, k) * x1;
    if (k + 2 < s) v -= AT(du2, k) * x2;
    v /= AT(dg, k);
    if (fabs(v) > big) {
      const R sm = R(1) / big;
      for (int q = 0; q < s; ++q) AT(b, q) *= sm;
      v *= sm;
      x1 *= sm;
      x2 *= sm;
      nrm *= sm;
    }
    AT(b, k) = v;
    x2 = x1;
    x1 = v;
    nrm = fmax(nrm, fabs(v));
  }
  // normalise (scaled 2-norm)
  const R inv = nrm > R(0) ? R(1) / nrm : R(1);
  R ss = 0;
  for (int k = 0; k < s; ++k) {
    const R v = AT(b, k) * inv;
    ss += v * v;
  }
  const R f = ss > R(0) ? inv / sqrt(ss) : R(0);
  for (int k = 0; k < s; ++k) ZT[int64_t(j) * S + k] = AT(b, k) * f;
#undef AT
}

// Classical Gram-Schmidt with re-orthogonalisation inside each cluster, in
// ascending order: CTA b handles the cluster that starts at b.
template <typename R>
__global__ void __launch_bounds__(256) cluster_cgs_kernel(int s, const int* __restrict__ cstart,
                                                          R* __restrict__ ZT) {
  const int b = blockIdx.x;
  if (cstart[b] != b) return;
  int end = b + 1;
  while (end < s && cstart[end] == b) ++end;
  if (end - b == 1) return;
  extern __shared__ unsigned char shc[];
  R* x = reinterpret_cast<R*>(shc);  // s
  R* c = x + s;                      // cluster size
  __shared__ R red[8];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t S = s;
  for (int j = b + 1; j < end; ++j) {
    for (int r = t; r < s; r += blockDim.x) x[r] = ZT[int64_t(j) * S + r];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = b + warp; i < j; i += blockDim.x / 32) {
        const R* q = ZT + int64_t(i) * S;
        R acc = 0;
        for (int r = lane; r < s; r += 32) acc += q[r] * x[r];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) c[i - b] = acc;
      }
      __syncthreads();
      for (int r = t; r < s; r += blockDim.x) {
        R acc = 0;
        for (int i = b; i < j; ++i) acc += c[i - b] * ZT[int64_t(i) * S + r];
        x[r] -= acc;
      }
      __syncthreads();
    }
    R part = 0;
    for (int r = t; r < s; r += blockDim.x) part += x[r] * x[r];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    R nn = 0;
    for (int w = 0; w < 8; ++w) nn += red[w];
    if (nn > R(0)) {
      const R f = R(1) / sqrt(nn);
      for (int r = t; r < s; r += blockDim.x) ZT[int64_t(j) * S + r] = x[r] * f;
    }  // else: the vector lay in the span of the earlier ones; keep it as it was
    __syncthreads();
  }
}

// rank[c] = position of d[c] in ascending order (ties by index)
template <typename R>
__global__ void rank_kernel(int s, const R* __restrict__ d, int* __restrict__ rank, double* __restrict__ lam) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const R v = d[c];
  int r = 0;
  for (int k = 0; k < s; ++k) {
    const R u = d[k];
    r += (u < v) || (u == v && k < c);
  }
  rank[c] = r;
  if (lam) lam[r] = double(v);
}

// Z_T = I G_1 G_2 ..., one thread per row, rows kept in shared memory as
// [col][row]; the new z_i of a rotation chain is carried in a register.
template <typename R>
__global__ void rot_accum_kernel(int s, int rpb, const int* __restrict__ ri, const R* __restrict__ rc,
                                 const R* __restrict__ rs, const int64_t* __restrict__ nrot, R* __restrict__ ZTc) {
  extern __shared__ unsigned char shraw[];
  R* zs = reinterpret_cast<R*>(shraw);  // s * rpb
  const int r0 = blockIdx.x * rpb;
  for (int idx = threadIdx.x; idx < s * rpb; idx += blockDim.x) {
    const int c = idx / rpb, rr = idx % rpb;
    zs[idx] = (r0 + rr == c) ? R(1) : R(0);
  }
  __syncthreads();
  const int64_t nr = *nrot;
  const int t = threadIdx.x;
  if (t < rpb) {
    int prev = -2;
    R carry = 0;
    for (int64_t q = 0; q < nr; ++q) {
      const int i = __ldg(ri + q);
      const R c = __ldg(rc + q), sn = __ldg(rs + q);
      R b;
      if (i + 1 == prev) {
        b = carry;
      } else {
        if (prev >= 0) zs[prev * rpb + t] = carry;
        b = zs[(i + 1) * rpb + t];
      }
      const R a = zs[i * rpb + t];
      zs[(i + 1) * rpb + t] = sn * a + c * b;
      carry = c * a - sn * b;
      prev = i;
    }
    if (prev >= 0) zs[prev * rpb + t] = carry;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < s * rpb; idx += blockDim.x) {
    const int c = idx / rpb, rr = idx % rpb;
    const int row = r0 + rr;
    if (row < s) ZTc[int64_t(c) * s + row] = zs[idx];
  }
}

// Z(:, rank[j]) = H_0 ... H_{s-3} Z_T(:, j); one warp per vector.  Output in
// float64 (Zd, leading dimension ldz).
template <typename R>
__global__ void __launch_bounds__(256) backtrans_kernel(int s, int wpb, const R* __restrict__ Vh,
                                                        const R* __restrict__ tau, const R* __restrict__ ZTc,
                                                        const int* __restrict__ rank, double* __restrict__ Zd,
                                                        int64_t ldz) {
  extern __shared__ unsigned char shraw[];
  R* zw = reinterpret_cast<R*>(shraw);  // wpb warps x s
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * wpb + warp;
  if (j >= s) return;
  R* z = zw + int64_t(warp) * s;
  for (int i = lane; i < s; i += 32) z[i] = ZTc[int64_t(j) * s + i];
  __syncwarp();
  for (int k = s - 3; k >= 0; --k) {
    const R tk = tau[k];
    if (tk == R(0)) continue;
    const R* v = Vh + int64_t(k) * s;
    R dot = 0;
    for (int i = k + 1 + lane; i < s; i += 32) dot += v[i] * z[i];
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    const R f = tk * dot;
    for (int i = k + 1 + lane; i < s; i += 32) z[i] -= f * v[i];
    __syncwarp();
  }
  const int col = rank[j];
  for (int i = lane; i < s; i += 32) Zd[int64_t(i) * ldz + col] = double(z[i]);
}

template <typename R>
struct QLWork {
  R *Wm, *Vh, *ZT, *tau, *d, *e, *p, *rc, *rs;
  int *ri, *rank, *status;
  int64_t* nrot;
  int64_t cap;
};

struct Carver {
  char* c;
  explicit Carver(void* base) : c(static_cast<char*>(base)) {}
  template <typename T>
  T* take(size_t n) {
    T* r = reinterpret_cast<T*>(c);
    c += (n * sizeof(T) + 255) & ~size_t(255);
    return r;
  }
};

template <typename R>
size_t ql_work_bytes(int s) {
  const size_t ss = size_t(s) * s, cap = 8 * ss + 1024;
  return 3 * (ss * sizeof(R) + 256) + 4 * (size_t(s) * sizeof(R) + 256) + 2 * (cap * sizeof(R) + 256) +
         (cap * sizeof(int) + 256) + (size_t(s) * sizeof(int) + 256) + 512;
}

template <typename R>
QLWork<R> ql_carve(int s, Carver& cv) {
  QLWork<R> w;
  const size_t ss = size_t(s) * s;
  w.cap = int64_t(8 * ss + 1024);
  w.Wm = cv.take<R>(ss);
  w.Vh = cv.take<R>(ss);
  w.ZT = cv.take<R>(ss);
  w.tau = cv.take<R>(s);
  w.d = cv.take<R>(s);
  w.e = cv.take<R>(s);
  w.p = cv.take<R>(s);
  w.rc = cv.take<R>(w.cap);
  w.rs = cv.take<R>(w.cap);
  w.ri = cv.take<int>(w.cap);
  w.rank = cv.take<int>(s);
  w.status = cv.take<int>(4);
  w.nrot = cv.take<int64_t>(2);
  return w;
}

// bisection + inverse iteration in precision R: eigenvectors of T into
// w.ZT (column j = eigenvector of the j-th smallest eigenvalue), ranks
// (identity) and eigenvalues (float64, if lam)
template <typename R>
static cudaError_t tri_invit(int s, QLWork<R>& w, double* lam, cudaStream_t st) {
  const size_t ss = size_t(s) * s;
  R* dl = w.rc;
  R* dgv = w.rc + ss;
  R* du = w.rc + 2 * ss;
  R* du2 = w.rc + 3 * ss;
  R* bv = w.rc + 4 * ss;
  R* lamr = w.rs;
  R* sig = w.rs + s;
  R* pert = w.rs + 2 * s;
  int* cstart = reinterpret_cast<int*>(w.rs + 2 * s + 64);
  unsigned char* piv = reinterpret_cast<unsigned char*>(w.ri);
  const unsigned nb = (unsigned)cdiv(s, 128);
  bisect_kernel<R><<<(unsigned)cdiv(s, 4), 128, 2 * size_t(s) * sizeof(R), st>>>(s, w.d, w.e, lamr);
  count_launches(1);
  invit_prep_kernel<R><<<1, 32, 0, st>>>(s, w.d, w.e, lamr, sig, cstart, pert); count_launches(1);
  cudaFuncSetAttribute(cluster_cgs_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  for (int pass = 0; pass < 2; ++pass) {
    invit_kernel<R><<<nb, 128, 0, st>>>(s, w.d, w.e, sig, pert, dl, dgv, du, du2, piv, bv, w.ZT, pass);
    count_launches(1);
    cluster_cgs_kernel<R><<<s, 256, 2 * size_t(s) * sizeof(R), st>>>(s, cstart, w.ZT); count_launches(1);
  }
  rank_kernel<R><<<nb, 128, 0, st>>>(s, lamr, w.rank, lam); count_launches(1);
  return cudaGetLastError();
}

// Stage 1 in precision R: eigenvalues (ascending) into lam (if non-null) and
// eigenvectors (float64, columns in ascending order) into Zd.
template <typename R>
cudaError_t ql_eig(int s, const double* A, int64_t lda, double* lam, double* Zd, int64_t ldz, QLWork<R>& w,
                   int* status_dev, cudaStream_t st, bool invit) {
  const int64_t ss = int64_t(s) * s;
  copy_sym_kernel<R><<<(unsigned)cdiv(ss, 256), 256, 0, st>>>(s, A, lda, w.Wm); count_launches(1);
  if (s >= 3) {
    int nb = (s + 7) / 8;
    if (nb > num_sms()) nb = num_sms();
    const size_t shm = 2 * size_t(s) * sizeof(R);
    cudaFuncSetAttribute(sytrd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sytrd_kernel<R>, 256, shm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int sv = s;
    void* args[] = {&sv, &w.Wm, &w.Vh, &w.tau, &w.d, &w.e, &w.p};
    cudaError_t err = cudaLaunchCooperativeKernel((void*)sytrd_kernel<R>, dim3(nb), dim3(256), args, shm, st);
    count_launches(1);
    if (err != cudaSuccess) return err;
  } else {
    small_tridiag_kernel<R><<<1, 32, 0, st>>>(s, w.Wm, w.d, w.e, w.tau); count_launches(1);
  }
  cudaFuncSetAttribute(backtrans_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (invit) {
    if (cudaError_t err = tri_invit(s, w, lam, st)) return err;
  } else {
    cudaFuncSetAttribute(tql_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    tql_kernel<R><<<1, 32, 2 * size_t(s) * sizeof(R), st>>>(s, w.d, w.e, w.ri, w.rc, w.rs, w.cap, w.nrot,
                                                            status_dev ? status_dev : w.status); count_launches(1);
    rank_kernel<R><<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.d, w.rank, lam); count_launches(1);
    int rpb = 32;
    while (rpb > 1 && size_t(s) * rpb * sizeof(R) > 200 * 1024) rpb >>= 1;
    cudaFuncSetAttribute(rot_accum_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    rot_accum_kernel<R><<<(unsigned)cdiv(s, rpb), 64, size_t(s) * rpb * sizeof(R), st>>>(s, rpb, w.ri, w.rc, w.rs,
                                                                                         w.nrot, w.ZT); count_launches(1);
  }
  int wpb = 8;
  while (wpb > 1 && size_t(wpb) * s * sizeof(R) > 200 * 1024) --wpb;
  backtrans_kernel<R><<<(unsigned)cdiv(s, wpb), 32 * wpb, size_t(wpb) * s * sizeof(R), st>>>(
      s, wpb, w.Vh, w.tau, w.ZT, w.rank, Zd, ldz); count_launches(1);
  return cudaGetLastError();
}

size_t syev_qr64_work_bytes(int s) { return ql_work_bytes<double>(s); }

cudaError_t syev_qr64(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                      int* status_dev, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  Carver cv(work);
  QLWork<double> w = ql_carve<double>(s, cv);
  return ql_eig<double>(s, A, lda, lam, Z, ldz, w, status_dev, st, false);
}


// ---------------------------------------------------------------------------
// stage 2: Ogita-Aishima refinement in double-float arithmetic
// ---------------------------------------------------------------------------
constexpr int OA_ITERS = 5;
constexpr int MAX_CLUSTER = 48;  // two 48 x 48 float64 blocks fit in static shared memory

// lambda_i = S_ii / G_ii (G = X^T X, so 1 - R_ii = G_ii)
__global__ void oa_lambda_kernel(int s, const double* __restrict__ G, const double* __restrict__ S,
                                 double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) lam[i] = S[int64_t(i) * s + i] / G[int64_t(i) * s + i];
}

// Clusters: consecutive lam (ascending up to the refinement's changes) whose
// gaps are at most tau = tau_rel * max |lam|.  cid[i] = first index of i's
// cluster.  One thread (s sequential comparisons).
__global__ void cluster_kernel(int s, const double* __restrict__ lam, double tau_rel, int* __restrict__ cid,
                               int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0.0;
  for (int i = 0; i < s; ++i) mx = fmax(mx, fabs(lam[i]));
  const double tau = tau_rel * mx;
  int start = 0, worst = 1;
  cid[0] = 0;
  for (int i = 1; i < s; ++i) {
    if (fabs(lam[i] - lam[i - 1]) <= tau) {
      cid[i] = start;
    } else {
      start = i;
      cid[i] = i;
    }
    worst = max(worst, i - start + 1);
  }
  if (worst > MAX_CLUSTER) *status = 3;
}

// E = correction of the Ogita-Aishima step (float64, s x s row-major)
__global__ void oa_e_kernel(int s, const double* __restrict__ G, const double* __restrict__ S,
                            const double* __restrict__ lam, const int* __restrict__ cid, double* __restrict__ E) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(s) * s) return;
  const int i = int(idx / s), j = int(idx % s);
  const double Rij = (i == j ? 1.0 : 0.0) - G[idx];
  if (cid[i] == cid[j]) {
    E[idx] = 0.5 * Rij;
  } else {
    E[idx] = (S[idx] + lam[j] * Rij) / (lam[j] - lam[i]);
  }
}

// Cyclic Jacobi on each cluster block of S (one warp per cluster): writes the
// block rotation V_C into Q (s x s, identity elsewhere) and the block's
// eigenvalues into lam.
__global__ void cluster_jacobi_kernel(int s, const double* __restrict__ S, const int* __restrict__ cid,
                                      double* __restrict__ Q, double* __restrict__ lam) {
  __shared__ double a[MAX_CLUSTER * MAX_CLUSTER];
  __shared__ double v[MAX_CLUSTER * MAX_CLUSTER];
  __shared__ double cs[2];
  const int start = blockIdx.x;
  if (start >= s || cid[start] != start) return;
  int m = 1;
  while (start + m < s && cid[start + m] == start) ++m;
  if (m == 1 || m > MAX_CLUSTER) return;
  const int lane = threadIdx.x;
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    a[idx] = 0.5 * (S[int64_t(start + i) * s + start + j] + S[int64_t(start + j) * s + start + i]);
    v[idx] = i == j ? 1.0 : 0.0;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, nrm = 0.0;
    for (int idx = lane; idx < m * m; idx += 32) {
      const int i = idx / m, j = idx % m;
      nrm += a[idx] * a[idx];
      if (i != j) off += a[idx] * a[idx];
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    if (off <= 1e-32 * nrm || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        if (lane == 0) {
          const double apq = a[p * m + q];
          double c = 1.0, sn = 0.0;
          if (fabs(apq) > 1e-300) {
            const double theta = (a[q * m + q] - a[p * m + p]) / (2.0 * apq);
            const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sn = t * c;
          }
          cs[0] = c;
          cs[1] = sn;
        }
        __syncwarp();
        const double c = cs[0], sn = cs[1];
        if (sn != 0.0) {
          // columns p, q of a and v
          for (int r = lane; r < m; r += 32) {
            const double ap = a[r * m + p], aq = a[r * m + q];
            a[r * m + p] = c * ap - sn * aq;
            a[r * m + q] = sn * ap + c * aq;
            const double vp = v[r * m + p], vq = v[r * m + q];
            v[r * m + p] = c * vp - sn * vq;
            v[r * m + q] = sn * vp + c * vq;
          }
          __syncwarp();
          // rows p, q of a
          for (int r = lane; r < m; r += 32) {
            const double ap = a[p * m + r], aq = a[q * m + r];
            a[p * m + r] = c * ap - sn * aq;
            a[q * m + r] = sn * ap + c * aq;
          }
        }
        __syncwarp();
      }
    }
  }
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    Q[int64_t(start + i) * s + start + j] = v[idx];
  }
  for (int i = lane; i < m; i += 32) lam[start + i] = a[i * m + i];
}

__global__ void eye_kernel(int s, double* __restrict__ Q) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx < int64_t(s) * s) Q[idx] = (idx / s == idx % s) ? 1.0 : 0.0;
}


__device__ __forceinline__ double elem_value(const dd& x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ double elem_value(const double& x) { return x; }

// Z(:, rank[j]) = X(:, j), lam_out[rank[j]] = lam[j]
template <typename T>
__global__ void permute_kernel(int s, const T* __restrict__ X, const int* __restrict__ rank,
                               const double* __restrict__ lam, double* __restrict__ Z, int64_t ldz,
                               double* __restrict__ lam_out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(s) * s) return;
  const int i = int(idx / s), j = int(idx % s);
  Z[int64_t(i) * ldz + rank[j]] = elem_value(X[idx]);
  if (i == 0) lam_out[rank[j]] = lam[j];
}

// refinement work for blocks of element type T (double-float or float64)
template <typename T>
struct RefWork {
  double *Zd, *G, *S, *E, *Q, *lam, *scr;
  T *Add, *X, *X2, *AX, *Cs;
  int* cid;
  int* rank;
};

template <typename T>
static size_t ref_bytes(int s) {
  const size_t ss = size_t(s) * s;
  const size_t scr = gram_scratch_elems(s, s, s, true);
  return 5 * (ss * 8 + 256) + (size_t(s) * 8 + 256) + (scr * 8 + 256) + 5 * (ss * sizeof(T) + 256) +
         2 * (size_t(s) * 4 + 256) + 1024;
}

template <typename T>
static RefWork<T> ref_carve(int s, Carver& cv) {
  RefWork<T> w;
  const size_t ss = size_t(s) * s;
  w.Zd = cv.take<double>(ss);
  w.G = cv.take<double>(ss);
  w.S = cv.take<double>(ss);
  w.E = cv.take<double>(ss);
  w.Q = cv.take<double>(ss);
  w.lam = cv.take<double>(s);
  w.scr = cv.take<double>(gram_scratch_elems(s, s, s, true));
  w.Add = cv.take<T>(ss);
  w.X = cv.take<T>(ss);
  w.X2 = cv.take<T>(ss);
  w.AX = cv.take<T>(ss);
  w.Cs = cv.take<T>(ss);
  w.cid = cv.take<int>(s);
  w.rank = cv.take<int>(s);
  return w;
}

size_t syev_work_bytes(int s) { return ql_work_bytes<float>(s) + ref_bytes<dd>(s) + 512; }
size_t syev64_work_bytes(int s) { return ql_work_bytes<double>(s) + ref_bytes<double>(s) + 512; }

template <typename T>
static Blk<T> sq(T* p, int s) {
  Blk<T> b;
  b.add(p, s, s);
  return b;
}

constexpr int dtype_of(Arith A) { return A == Arith::DF64 ? EIG_DF64 : EIG_F64; }

// G = X^T X, AX = A X, S = X^T A X for the current X (arithmetic A)
template <Arith A, typename T>
static cudaError_t oa_products(int s, RefWork<T>& w, cudaStream_t st) {
  cudaError_t e;
  if ((e = gram<A>(s, sq(w.X, s), sq(w.X, s), true, w.G, s, w.scr, st))) return e;
  if ((e = convert2d(s, s, w.X, s, dtype_of(A), w.Zd, s, EIG_F64, st))) return e;
  if ((e = stage_coef<A>(s, s, w.Zd, s, w.Cs, s, 1.0, st))) return e;
  if ((e = update<A>(s, sq(w.Add, s), w.Cs, s, sq(w.AX, s), 0.0, st))) return e;
  return gram<A>(s, sq(w.X, s), sq(w.AX, s), true, w.S, s, w.scr, st);
}

// Ogita-Aishima refinement of the eigenvector estimate in w.X (s x s,
// arithmetic A): `iters` corrections, clusters of Rayleigh quotients closer
// than tau_rel max |lam| diagonalised by Jacobi before each correction and at
// the end; eigenvalues ascending into lam, vectors into Z.  Inside a cluster
// the columns of X only span an approximate invariant subspace, so before
// each correction the cluster blocks of X^T A X are diagonalised and X
// rotated: otherwise the off-cluster corrections use Rayleigh quotients that
// are not eigenvalue estimates and the cluster subspace stops converging.
template <Arith A, typename T>
static cudaError_t refine(int s, RefWork<T>& w, int iters, double tau_rel, double* lam, double* Z, int64_t ldz,
                          int* status_dev, cudaStream_t st) {
  const int64_t ss = int64_t(s) * s;
  const unsigned gb = (unsigned)cdiv(ss, 256);
  cudaError_t e;
  for (int it = 0; it < iters; ++it) {
    if ((e = oa_products<A>(s, w, st))) return e;
    oa_lambda_kernel<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.G, w.S, w.lam); count_launches(1);
    if (it == 0) {
      cluster_kernel<<<1, 32, 0, st>>>(s, w.lam, tau_rel, w.cid, status_dev);
      count_launches(1);
    }
    eye_kernel<<<gb, 256, 0, st>>>(s, w.Q); count_launches(1);
    cluster_jacobi_kernel<<<s, 32, 0, st>>>(s, w.S, w.cid, w.Q, w.lam); count_launches(1);
    if ((e = stage_coef<A>(s, s, w.Q, s, w.Cs, s, 1.0, st))) return e;
    if ((e = update<A>(s, sq(w.X, s), w.Cs, s, sq(w.X2, s), 0.0, st))) return e;
    std::swap(w.X, w.X2);
    if ((e = oa_products<A>(s, w, st))) return e;
    oa_lambda_kernel<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.G, w.S, w.lam); count_launches(1);
    oa_e_kernel<<<gb, 256, 0, st>>>(s, w.G, w.S, w.lam, w.cid, w.E); count_launches(1);
    // X2 = X + X E
    if ((e = cudaMemcpyAsync(w.X2, w.X, sizeof(T) * ss, cudaMemcpyDeviceToDevice, st))) return e;
    if ((e = stage_coef<A>(s, s, w.E, s, w.Cs, s, 1.0, st))) return e;
    if ((e = update<A>(s, sq(w.X, s), w.Cs, s, sq(w.X2, s), 1.0, st))) return e;
    std::swap(w.X, w.X2);
  }
  // final: eigenvalues, cluster diagonalisation, ascending order
  if ((e = oa_products<A>(s, w, st))) return e;
  oa_lambda_kernel<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.G, w.S, w.lam); count_launches(1);
  if (iters == 0) {
    cluster_kernel<<<1, 32, 0, st>>>(s, w.lam, tau_rel, w.cid, status_dev);
    count_launches(1);
  }
  eye_kernel<<<gb, 256, 0, st>>>(s, w.Q); count_launches(1);
  cluster_jacobi_kernel<<<s, 32, 0, st>>>(s, w.S, w.cid, w.Q, w.lam); count_launches(1);
  if ((e = stage_coef<A>(s, s, w.Q, s, w.Cs, s, 1.0, st))) return e;
  if ((e = update<A>(s, sq(w.X, s), w.Cs, s, sq(w.X2, s), 0.0, st))) return e;
  rank_kernel<double><<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.lam, w.rank, nullptr); count_launches(1);
  permute_kernel<T><<<gb, 256, 0, st>>>(s, w.X2, w.rank, w.lam, Z, ldz, lam); count_launches(1);
  return cudaGetLastError();
}

// Double-float and mixed forms: float32 decomposition, OA_ITERS double-float
// refinement steps (clusters at 3e-6 max |lam|).
cudaError_t syev(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                 int* status_dev, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  Carver cv(work);
  QLWork<float> ql = ql_carve<float>(s, cv);
  RefWork<dd> w = ref_carve<dd>(s, cv);
  int* stat = status_dev ? status_dev : ql.status;
  cudaError_t e;
  if ((e = ql_eig<float>(s, A, lda, nullptr, w.Zd, s, ql, stat, st, true))) return e;
  if ((e = convert2d(s, s, w.Zd, s, EIG_F64, w.X, s, EIG_DF64, st))) return e;
  if ((e = convert2d(s, s, A, lda, EIG_F64, w.Add, s, EIG_DF64, st))) return e;
  return refine<Arith::DF64>(s, w, OA_ITERS, 3e-6, lam, Z, ldz, stat, st);
}

// Float64 form: float64 Householder tridiagonalisation, multisection
// bisection, inverse iteration with Gram-Schmidt inside clusters of nearly
// equal eigenvalues, back-transformation -- vectors accurate to about
// eps ||A|| / gap -- then one float64 Ogita-Aishima step on the library's
// float64 products, which squares that coupling away (clusters at 1e-10
// max |lam| diagonalised by Jacobi).
cudaError_t syev64(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                   int* status_dev, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  Carver cv(work);
  QLWork<double> ql = ql_carve<double>(s, cv);
  RefWork<double> w = ref_carve<double>(s, cv);
  int* stat = status_dev ? status_dev : ql.status;
  cudaError_t e;
  if ((e = ql_eig<double>(s, A, lda, nullptr, w.X, s, ql, stat, st, true))) return e;
  if ((e = cudaMemcpy2DAsync(w.Add, sizeof(double) * s, A, sizeof(double) * lda, sizeof(double) * s, s,
                             cudaMemcpyDeviceToDevice, st)))
    return e;
  return refine<Arith::F64>(s, w, 1, 1e-10, lam, Z, ldz, stat, st);
}

}  // namespace eig
