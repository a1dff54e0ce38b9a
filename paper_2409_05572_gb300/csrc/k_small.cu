// Small dense float64 kernels of the Rayleigh-Ritz and orthogonalisation
// steps (arXiv:2409.05572, Algorithms 1 and 3):
//   * Cholesky G = R^T R and R^{-1} for CholeskyQR (shifted variant of
//     Fukaya et al. 2020 on breakdown),
//   * symmetric eigensolver A = Z diag(lam) Z^T: Householder tridiagonal
//     reduction (grid-synchronised cooperative kernel), implicit QL with
//     Wilkinson shifts on the tridiagonal (Bowdler, Martin, Reinsch and
//     Wilkinson 1968) recording its Givens rotations, formation of the
//     Householder product, row-parallel application of the rotations, and an
//     ascending sort,
//   * the Householder QR and right-multiplication of the improved
//     Hetmaniuk-Lehoucq basis selection.
// These act on s x s matrices (s <= 3 k_max); they are latency / FP64-pipe
// bound and run on a few SMs.
#include <cooperative_groups.h>

#include <cstdio>

#include "small.cuh"

namespace cg = cooperative_groups;

namespace eig {

// ---------------------------------------------------------------------------
// Cholesky + triangular inverse, one CTA.
// status: 0 plain, 1 shifted, 2 broken down.
// ---------------------------------------------------------------------------
__device__ bool chol_upper_inplace(double* Rm, int w, int ld, const double* diag0, double* sh) {
  // Rm holds G (upper triangle used); on success its upper triangle is R.
  for (int j = 0; j < w; ++j) {
    if (threadIdx.x == 0) {
      const double d = Rm[j * ld + j];
      const double thr = 1e-14 * fmax(diag0[j], 0.0);
      if (!(d > thr) || !isfinite(d)) {
        sh[0] = -1.0;
      } else {
        sh[0] = sqrt(d);
        Rm[j * ld + j] = sh[0];
      }
    }
    __syncthreads();
    const double r = sh[0];
    if (r < 0.0) return false;
    for (int k = j + 1 + threadIdx.x; k < w; k += blockDim.x) Rm[j * ld + k] /= r;
    __syncthreads();
    const int m = w - j - 1;
    const int64_t tot = int64_t(m) * m;
    for (int64_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int i = j + 1 + int(idx / m), k = j + 1 + int(idx % m);
      if (k >= i) Rm[i * ld + k] -= Rm[j * ld + i] * Rm[j * ld + k];
    }
    __syncthreads();
  }
  return true;
}

__global__ void __launch_bounds__(512) chol_rinv_kernel(int w, int64_t nrows, const double* __restrict__ G,
                                                        int64_t ldg, double* __restrict__ Rinv,
                                                        double* __restrict__ work, int* status,
                                                        const int* gate, double u) {
  if (gate && *gate == 0) return;
  extern __shared__ double smem[];
  __shared__ double sh[2];
  const bool in_smem = (size_t(w) * w + w) * sizeof(double) <= 160 * 1024;
  double* Rm = in_smem ? smem : work;
  double* diag0 = in_smem ? smem + size_t(w) * w : work + size_t(w) * w;
  for (int64_t idx = threadIdx.x; idx < int64_t(w) * w; idx += blockDim.x) {
    const int i = int(idx / w), k = int(idx % w);
    Rm[idx] = G[i * ldg + k];
  }
  for (int i = threadIdx.x; i < w; i += blockDim.x) diag0[i] = G[i * ldg + i];
  __syncthreads();
  int st = 0;
  bool ok = chol_upper_inplace(Rm, w, w, diag0, sh);
  if (!ok) {
    // shifted CholeskyQR: G + s I, s = 11 (m w + w (w + 1)) u trace(G)
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int i = 0; i < w; ++i) tr += diag0[i];
      sh[1] = 11.0 * (double(nrows) * w + double(w) * (w + 1)) * u * tr;
    }
    __syncthreads();
    const double shift = sh[1];
    for (int64_t idx = threadIdx.x; idx < int64_t(w) * w; idx += blockDim.x) {
      const int i = int(idx / w), k = int(idx % w);
      Rm[idx] = G[i * ldg + k] + (i == k ? shift : 0.0);
    }
    __syncthreads();
    ok = chol_upper_inplace(Rm, w, w, diag0, sh);
    st = ok ? 1 : 2;
  }
  if (!ok) {
    if (threadIdx.x == 0) *status = 2;
    for (int64_t idx = threadIdx.x; idx < int64_t(w) * w; idx += blockDim.x)
      Rinv[idx] = (idx / w == idx % w) ? 1.0 : 0.0;
    return;
  }
  // R^{-1}, column by column: Rinv[i][j] = -(sum_{k=i}^{j-1} Rinv[i][k] R[k][j]) / R[j][j]
  for (int64_t idx = threadIdx.x; idx < int64_t(w) * w; idx += blockDim.x) Rinv[idx] = 0.0;
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    const double rjj = Rm[j * w + j];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      if (i == j) {
        Rinv[j * w + j] = 1.0 / rjj;
      } else {
        double s = 0.0;
        for (int k = i; k < j; ++k) s += Rinv[i * w + k] * Rm[k * w + j];
        Rinv[i * w + j] = -s / rjj;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *status = st;
}

cudaError_t chol_rinv(int w, int64_t nrows, const double* G, int64_t ldg, double* Rinv, double* work,
                      int* status, cudaStream_t st, const int* gate, double unit_round) {
  const size_t need = (size_t(w) * w + w) * sizeof(double);
  const size_t shm = need <= 160 * 1024 ? need : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(chol_rinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  chol_rinv_kernel<<<1, 512, shm, st>>>(w, nrows, G, ldg, Rinv, work, status, gate, unit_round);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation (cooperative).  Wm: working copy of A
// (s x s row-major, both triangles), Vh: reflector k in row k (entries
// k+1..s-1), tau[k]; d, e: diagonal and subdiagonal of T = Q^T A Q with
// Q = H_0 H_1 ... H_{s-3}, H_k = I - tau_k v_k v_k^T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red) {
  // 256-thread block reduction; all threads get the result
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < 8; ++i) t += red[i];
  return t;
}

__global__ void __launch_bounds__(256) sytrd_kernel(int s, double* __restrict__ Wm, double* __restrict__ Vh,
                                                    double* __restrict__ tau, double* __restrict__ d,
                                                    double* __restrict__ e, double* __restrict__ p) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sh[];  // vsh[s], psh[s]
  double* vsh = sh;
  double* psh = sh + s;
  __shared__ double red[8];
  const int nb = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int gw = b * 8 + warp, nw = nb * 8;
  for (int k = 0; k + 2 < s; ++k) {
    const int m = s - k - 1;  // x = A[k+1:, k] = A[k, k+1:] (symmetric storage)
    const double* rowk = Wm + int64_t(k) * s + (k + 1);
    double part = 0.0, part_tail = 0.0;
    for (int i = t; i < m; i += blockDim.x) {
      const double x = rowk[i];
      vsh[i] = x;
      part += x * x;
      if (i > 0) part_tail += x * x;
    }
    const double nrm2 = block_sum(part, red);
    const double tail2 = block_sum(part_tail, red);
    const double x0 = vsh[0];
    double tk, alpha;
    if (tail2 == 0.0) {
      tk = 0.0;
      alpha = x0;
    } else {
      const double nrm = sqrt(nrm2);
      alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      tk = 2.0 / (tail2 + v0 * v0);
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
    if (tk != 0.0) {
      // p = tau W_sub v: one warp per row, lanes along the row
      for (int i = gw; i < m; i += nw) {
        const double* wr = Wm + int64_t(k + 1 + i) * s + (k + 1);
        double acc = 0.0;
        for (int j = lane; j < m; j += 32) acc += wr[j] * vsh[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) p[i] = tk * acc;
      }
    }
    grid.sync();
    if (tk != 0.0) {
      double pv = 0.0;
      for (int i = t; i < m; i += blockDim.x) {
        const double pi = p[i];
        psh[i] = pi;
        pv += pi * vsh[i];
      }
      const double K = 0.5 * tk * block_sum(pv, red);
      // rank-2 update W -= v w^T + w v^T, w = p - K v; one warp per row
      for (int i = gw; i < m; i += nw) {
        const double vi = vsh[i];
        const double wi = psh[i] - K * vi;
        double* wr = Wm + int64_t(k + 1 + i) * s + (k + 1);
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
    e[s - 1] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Implicit QL with Wilkinson shifts on the symmetric tridiagonal (d, e),
// e[i] = T[i+1][i].  One thread.  Every Givens rotation applied to the
// eigenvector columns (i, i+1) is appended to (ri, rc, rs):
//   z_i <- c z_i - s z_{i+1},  z_{i+1} <- s z_i + c z_{i+1}.
// ---------------------------------------------------------------------------
__global__ void tql_kernel(int s, double* __restrict__ dg, double* __restrict__ eg, int* __restrict__ ri,
                           double* __restrict__ rc, double* __restrict__ rs, int64_t cap,
                           int64_t* nrot, int* status) {
  // d and e live in shared memory while the single thread iterates: the
  // rotation chain is latency bound and global round trips would dominate.
  extern __shared__ double de[];
  double* d = de;
  double* e = de + s;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    d[i] = dg[i];
    e[i] = eg[i];
  }
  __syncthreads();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double eps = 2.220446049250313e-16;
  int64_t cnt = 0;
  int st = 0;
  e[s - 1] = 0.0;
  for (int l = 0; l < s && st == 0; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m < s - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) {
        st = 1;
        break;
      }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      double sn = 1.0, cs = 1.0, p = 0.0;
      bool early = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = sn * e[i];
        const double bb = cs * e[i];
        const double hh = f * f + g * g;
        double rinv;
        if (hh > 1e-280 && hh < 1e280) {
          rinv = rsqrt(hh);
          r = hh * rinv;
        } else {
          r = hypot(f, g);
          rinv = r != 0.0 ? 1.0 / r : 0.0;
        }
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          early = true;
          break;
        }
        sn = f * rinv;
        cs = g * rinv;
        g = d[i + 1] - p;
        r = (d[i] - g) * sn + 2.0 * cs * bb;
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
      e[m] = 0.0;
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

// rank[c] = position of d[c] in ascending order (ties by index); lam sorted
__global__ void rank_kernel(int s, const double* __restrict__ d, int* __restrict__ rank,
                            double* __restrict__ lam) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const double v = d[c];
  int r = 0;
  for (int k = 0; k < s; ++k) {
    const double u = d[k];
    r += (u < v) || (u == v && k < c);
  }
  rank[c] = r;
  lam[r] = v;
}

// Eigenvectors of T: Z_T = I G_1 G_2 ..., one thread per row (RPB rows per
// CTA kept in shared memory as [col][row]); written column-major (ZTc[j][i]).
__global__ void rot_accum_kernel(int s, int rpb, const int* __restrict__ ri, const double* __restrict__ rc,
                                 const double* __restrict__ rs, const int64_t* __restrict__ nrot,
                                 double* __restrict__ ZTc) {
  extern __shared__ double zs[];  // s * rpb
  const int r0 = blockIdx.x * rpb;
  for (int idx = threadIdx.x; idx < s * rpb; idx += blockDim.x) {
    const int c = idx / rpb, rr = idx % rpb;
    zs[idx] = (r0 + rr == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int64_t nr = *nrot;
  const int t = threadIdx.x;
  if (t < rpb) {
    // Within a QL sweep consecutive rotations act on (i, i+1) then
    // (i-1, i): the new z_i is carried in a register instead of a shared
    // memory round trip.
    int prev = -2;
    double carry = 0.0;
    for (int64_t q = 0; q < nr; ++q) {
      const int i = __ldg(ri + q);
      const double c = __ldg(rc + q), sn = __ldg(rs + q);
      double b;
      if (i + 1 == prev) {
        b = carry;
      } else {
        if (prev >= 0) zs[prev * rpb + t] = carry;
        b = zs[(i + 1) * rpb + t];
      }
      const double a = zs[i * rpb + t];
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

// Z(:, rank[j]) = H_0 H_1 ... H_{s-3} Z_T(:, j): one warp per eigenvector,
// the vector in shared memory, lanes along the reflector.
__global__ void __launch_bounds__(256) backtrans_kernel(int s, int wpb, const double* __restrict__ Vh,
                                                        const double* __restrict__ tau,
                                                        const double* __restrict__ ZTc,
                                                        const int* __restrict__ rank, double* __restrict__ Z,
                                                        int64_t ldz) {
  extern __shared__ double zw[];  // wpb warps x s
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * wpb + warp;
  if (j >= s) return;
  double* z = zw + int64_t(warp) * s;
  for (int i = lane; i < s; i += 32) z[i] = ZTc[int64_t(j) * s + i];
  __syncwarp();
  for (int k = s - 3; k >= 0; --k) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const double* v = Vh + int64_t(k) * s;
    double dot = 0.0;
    for (int i = k + 1 + lane; i < s; i += 32) dot += v[i] * z[i];
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    const double f = tk * dot;
    for (int i = k + 1 + lane; i < s; i += 32) z[i] -= f * v[i];
    __syncwarp();
  }
  const int col = rank[j];
  for (int i = lane; i < s; i += 32) Z[int64_t(i) * ldz + col] = z[i];
}

__global__ void small_tridiag_kernel(int s, const double* Wm, double* d, double* e, double* tau) {
  if (threadIdx.x != 0) return;
  d[0] = Wm[0];
  e[0] = 0.0;
  tau[0] = 0.0;
  if (s == 2) {
    d[1] = Wm[3];
    e[0] = Wm[2];
    e[1] = 0.0;
    tau[1] = 0.0;
  }
}

__global__ void copy_sym_kernel(int s, const double* __restrict__ A, int64_t lda, double* __restrict__ Wm) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(s) * s) return;
  const int i = int(idx / s), j = int(idx % s);
  // symmetrise: (A + A^T) / 2
  Wm[idx] = 0.5 * (A[int64_t(i) * lda + j] + A[int64_t(j) * lda + i]);
}

size_t syev_work_bytes(int s) {
  const size_t ss = size_t(s) * s;
  const size_t cap = 64 * ss + 1024;
  return (3 * ss + 6 * size_t(s)) * sizeof(double) + cap * (2 * sizeof(double) + sizeof(int)) +
         size_t(s) * sizeof(int) + 256;
}

struct SyevWork {
  double *Wm, *Vh, *Q, *tau, *d, *e, *p, *rc, *rs;
  int *ri, *rank, *status;
  int64_t* nrot;
  int64_t cap;
};

static SyevWork carve(int s, void* base) {
  SyevWork w;
  const size_t ss = size_t(s) * s;
  char* c = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    char* r = c;
    c += (bytes + 15) & ~size_t(15);
    return r;
  };
  w.cap = int64_t(64 * ss + 1024);
  w.Wm = (double*)take(ss * 8);
  w.Vh = (double*)take(ss * 8);
  w.Q = (double*)take(ss * 8);
  w.tau = (double*)take(size_t(s) * 8);
  w.d = (double*)take(size_t(s) * 8);
  w.e = (double*)take(size_t(s) * 8);
  w.p = (double*)take(size_t(s) * 8);
  w.rc = (double*)take(size_t(w.cap) * 8);
  w.rs = (double*)take(size_t(w.cap) * 8);
  w.ri = (int*)take(size_t(w.cap) * 4);
  w.rank = (int*)take(size_t(s) * 4);
  w.status = (int*)take(16);
  w.nrot = (int64_t*)take(16);
  return w;
}

cudaError_t syev(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                 int* status_dev, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  SyevWork w = carve(s, work);
  const int64_t ss = int64_t(s) * s;
  copy_sym_kernel<<<(unsigned)cdiv(ss, 256), 256, 0, st>>>(s, A, lda, w.Wm);
  if (s >= 3) {
    int nb = (s + 7) / 8;  // about one warp per row of the trailing matrix
    if (nb > num_sms()) nb = num_sms();
    const size_t shm = 2 * size_t(s) * sizeof(double);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(sytrd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sytrd_kernel, 256, shm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int sv = s;
    void* args[] = {&sv, &w.Wm, &w.Vh, &w.tau, &w.d, &w.e, &w.p};
    cudaError_t err = cudaLaunchCooperativeKernel((void*)sytrd_kernel, dim3(nb), dim3(256), args, shm, st);
    if (err != cudaSuccess) return err;
  } else {
    // s <= 2: the matrix is already tridiagonal and Q = I
    small_tridiag_kernel<<<1, 32, 0, st>>>(s, w.Wm, w.d, w.e, w.tau);
  }
  static bool attr3 = false;
  if (!attr3) {
    cudaFuncSetAttribute(tql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr3 = true;
  }
  tql_kernel<<<1, 32, 2 * size_t(s) * sizeof(double), st>>>(s, w.d, w.e, w.ri, w.rc, w.rs, w.cap, w.nrot,
                                                             status_dev ? status_dev : w.status);
  rank_kernel<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(s, w.d, w.rank, lam);
  int rpb = 32;
  while (rpb > 1 && size_t(s) * rpb * 8 > 200 * 1024) rpb >>= 1;
  static bool attr2 = false;
  if (!attr2) {
    cudaFuncSetAttribute(rot_accum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(backtrans_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    attr2 = true;
  }
  // w.Q holds Z_T column-major
  rot_accum_kernel<<<(unsigned)cdiv(s, rpb), 64, size_t(s) * rpb * 8, st>>>(s, rpb, w.ri, w.rc, w.rs, w.nrot,
                                                                              w.Q);
  int wpb = 8;
  while (wpb > 1 && size_t(wpb) * s * 8 > 200 * 1024) --wpb;
  backtrans_kernel<<<(unsigned)cdiv(s, wpb), 32 * wpb, size_t(wpb) * s * 8, st>>>(s, wpb, w.Vh, w.tau, w.Q, w.rank,
                                                                                 Z, ldz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Improved Hetmaniuk-Lehoucq basis selection.
// M = Z(nlock:nnow, nnow:s)^T  (m x q, m = s - nnow, q = nnow - nlock),
// Householder QR M = Q R (one CTA), then CP = Z(:, nnow:s) H_0 ... H_{q-1}
// restricted to its first q columns (one thread per row of Z).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) hl_qr_kernel(int s, int nnow, int nlock, const double* __restrict__ Z,
                                                    int64_t ldz, double* __restrict__ Mw,
                                                    double* __restrict__ htau) {
  const int m = s - nnow, q = nnow - nlock;
  __shared__ double red[256];
  const int t = threadIdx.x;
  // Mw (m x q row-major): Mw[i][j] = Z[nlock + j][nnow + i]
  for (int64_t idx = t; idx < int64_t(m) * q; idx += blockDim.x) {
    const int i = int(idx / q), j = int(idx % q);
    Mw[idx] = Z[int64_t(nlock + j) * ldz + nnow + i];
  }
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    // reflector for column k, rows k..m-1
    double part = 0.0;
    for (int i = k + 1 + t; i < m; i += blockDim.x) part += Mw[int64_t(i) * q + k] * Mw[int64_t(i) * q + k];
    red[t] = part;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (t < o) red[t] += red[t + o];
      __syncthreads();
    }
    const double tail2 = red[0];
    __syncthreads();
    const double x0 = Mw[int64_t(k) * q + k];
    double tk = 0.0;
    if (tail2 != 0.0) {
      const double nrm = sqrt(x0 * x0 + tail2);
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      tk = 2.0 / (tail2 + v0 * v0);
      __syncthreads();
      if (t == 0) Mw[int64_t(k) * q + k] = v0;  // v stored in column k (rows k..), v0 at the top
    }
    if (t == 0) htau[k] = tk;
    __syncthreads();
    if (tk != 0.0) {
      // apply H_k to columns k+1..q-1: col -= tk v (v^T col)
      for (int j = k + 1 + t; j < q; j += blockDim.x) {
        double dot = 0.0;
        for (int i = k; i < m; ++i) dot += Mw[int64_t(i) * q + k] * Mw[int64_t(i) * q + j];
        const double f = tk * dot;
        for (int i = k; i < m; ++i) Mw[int64_t(i) * q + j] -= f * Mw[int64_t(i) * q + k];
      }
    }
    __syncthreads();
  }
}

// CP[row][0:q] = (Z(row, nnow:s) H_0 ... H_{q-1})[0:q]
__global__ void hl_apply_kernel(int s, int nnow, int nlock, const double* __restrict__ Z, int64_t ldz,
                                const double* __restrict__ Mw, const double* __restrict__ htau,
                                double* __restrict__ CP, int64_t ldcp, double* __restrict__ rowbuf) {
  const int m = s - nnow, q = nnow - nlock;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= s) return;
  double* z = rowbuf + int64_t(row) * m;
  for (int i = 0; i < m; ++i) z[i] = Z[int64_t(row) * ldz + nnow + i];
  for (int k = 0; k < q; ++k) {
    const double tk = htau[k];
    if (tk == 0.0) continue;
    double dot = 0.0;
    for (int i = k; i < m; ++i) dot += z[i] * Mw[int64_t(i) * q + k];
    const double f = tk * dot;
    for (int i = k; i < m; ++i) z[i] -= f * Mw[int64_t(i) * q + k];
  }
  for (int j = 0; j < q; ++j) CP[int64_t(row) * ldcp + j] = z[j];
}

size_t hl_work_bytes(int s, int nnow, int nlock) {
  const size_t m = size_t(s - nnow), q = size_t(nnow - nlock);
  return (m * q + q + size_t(s) * m) * sizeof(double) + 64;
}

cudaError_t hl_trick(int s, int nnow, int nlock, const double* Z, int64_t ldz, double* CP, int64_t ldcp,
                     void* work, cudaStream_t st) {
  const int m = s - nnow, q = nnow - nlock;
  if (q <= 0) return cudaSuccess;
  if (m < q) return cudaErrorInvalidValue;
  double* Mw = static_cast<double*>(work);
  double* htau = Mw + size_t(m) * q;
  double* rowbuf = htau + q;
  hl_qr_kernel<<<1, 256, 0, st>>>(s, nnow, nlock, Z, ldz, Mw, htau);
  hl_apply_kernel<<<(unsigned)cdiv(s, 64), 64, 0, st>>>(s, nnow, nlock, Z, ldz, Mw, htau, CP, ldcp, rowbuf);
  return cudaGetLastError();
}

}  // namespace eig
