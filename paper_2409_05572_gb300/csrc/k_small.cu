// Small dense float64 kernels of the Rayleigh-Ritz and orthogonalisation
// steps (arXiv:2409.05572, Algorithms 1 and 3):
//   * Cholesky G = R^T R and R^{-1} for CholeskyQR (shifted variant of
//     Fukaya et al. 2020 on breakdown),
//   * the Householder QR and right-multiplication of the improved
//     Hetmaniuk-Lehoucq basis selection.
// These act on s x s matrices (s <= 3 k_max); they are latency / FP64-pipe
// bound and run on a few SMs.
#include <cstdio>

#include "small.cuh"

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
  chol_rinv_kernel<<<1, 512, shm, st>>>(w, nrows, G, ldg, Rinv, work, status, gate, unit_round); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation (cooperative).  Wm: working copy of A
// (s x s row-major, both triangles), Vh: reflector k in row k (entries
// k+1..s-1), tau[k]; d, e: diagonal and subdiagonal of T = Q^T A Q with
// Q = H_0 H_1 ... H_{s-3}, H_k = I - tau_k v_k v_k^T.
// ---------------------------------------------------------------------------
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
  hl_qr_kernel<<<1, 256, 0, st>>>(s, nnow, nlock, Z, ldz, Mw, htau); count_launches(1);
  hl_apply_kernel<<<(unsigned)cdiv(s, 64), 64, 0, st>>>(s, nnow, nlock, Z, ldz, Mw, htau, CP, ldcp, rowbuf); count_launches(1);
  return cudaGetLastError();
}

}  // namespace eig
