// Small dense float64 kernels of the Rayleigh-Ritz and orthogonalisation
// steps (arXiv:2409.05572, Algorithms 1 and 3):
//   * Cholesky G = R^T R and R^{-1} for CholeskyQR (shifted variant of
//     Fukaya et al. 2020 on breakdown),
//   * the improved Hetmaniuk-Lehoucq basis selection (shifted CholeskyQR3 of
//     a block of Z and the product with Z, built from the float64 Gram,
//     Cholesky and update kernels).
// These act on s x s matrices (s <= 3 k_max); they are latency / FP64-pipe
// bound.
#include <cstdio>

#include <utility>

#include "blocks.cuh"
#include "small.cuh"

namespace eig {

// ---------------------------------------------------------------------------
// Cholesky + triangular inverse, one CTA.
// status: 0 plain, 1 shifted, 2 broken down.
// ---------------------------------------------------------------------------
__device__ bool chol_upper_inplace(double* Rm, int w, int ld, const double* diag0, double* sh) {
  // Rm holds G (upper triangle used); on success its upper triangle is R.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
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
    // trailing update of the upper triangle: warps over rows, lanes over columns
    for (int i = j + 1 + warp; i < w; i += nw) {
      const double rji = Rm[j * ld + i];
      for (int k = i + lane; k < w; k += 32) Rm[i * ld + k] -= rji * Rm[j * ld + k];
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
  const bool in_smem = (size_t(w) * w + 2 * size_t(w)) * sizeof(double) <= 160 * 1024;
  double* Rm = in_smem ? smem : work;
  double* diag0 = (in_smem ? smem : work) + size_t(w) * w;
  double* dinv = diag0 + w;
  for (int i = threadIdx.x >> 5; i < w; i += blockDim.x >> 5)
    for (int k = threadIdx.x & 31; k < w; k += 32) Rm[i * w + k] = G[i * ldg + k];
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
    for (int i = threadIdx.x >> 5; i < w; i += blockDim.x >> 5)
      for (int k = threadIdx.x & 31; k < w; k += 32) Rm[i * w + k] = G[i * ldg + k] + (i == k ? shift : 0.0);
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
  // R^{-1}: diagonal 1 / R_jj in dinv, Rinv[i][j] (i < j) kept in the free
  // lower triangle at Rm[j][i]; column j from the finished columns < j:
  // Rinv[i][j] = -(sum_{k=i}^{j-1} Rinv[i][k] R[k][j]) / R[j][j], one warp per i
  for (int j = threadIdx.x; j < w; j += blockDim.x) dinv[j] = 1.0 / Rm[j * w + j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 1; j < w; ++j) {
    for (int i = warp; i < j; i += nw) {
      double acc = 0.0;
      for (int k = i + lane; k < j; k += 32) acc += (k == i ? dinv[i] : Rm[k * w + i]) * Rm[k * w + j];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) Rm[j * w + i] = -acc * dinv[j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x >> 5; i < w; i += blockDim.x >> 5)
    for (int k = threadIdx.x & 31; k < w; k += 32)
      Rinv[i * w + k] = k == i ? dinv[i] : (k > i ? Rm[k * w + i] : 0.0);
  if (threadIdx.x == 0) *status = st;
}

cudaError_t chol_rinv(int w, int64_t nrows, const double* G, int64_t ldg, double* Rinv, double* work,
                      int* status, cudaStream_t st, const int* gate, double unit_round) {
  // Cholesky factor, first diagonal of G and 1 / R_jj (w^2 + 2w float64): in
  // shared memory when they fit, else in work (which must hold them)
  const size_t need = (size_t(w) * w + 2 * size_t(w)) * sizeof(double);
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
// Y = Z(nlock:nnow, nnow:s)^T  (m x q, m = s - nnow, q = nnow - nlock); its
// orthonormal QR factor Q by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa,
// Yamamoto and Yanagisawa, SISC 2020): three passes of G = Y^T Y (float64
// Gram), R^{-1} from the float64 Cholesky of G (shifted when G is not
// numerically positive definite), Y <- Y R^{-1}.  For a full-rank Y the thin
// Q factor is unique up to column signs, so this is the Householder Q of the
// same block up to signs, and the passes are float64 kernels over all SMs
// rather than q sequential reflector steps.  Then CP = Z(:, nnow:s) Q.
// ---------------------------------------------------------------------------
__global__ void hl_gather_kernel(int nnow, int nlock, int m, int q, const double* __restrict__ Z, int64_t ldz,
                                 double* __restrict__ Y) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(m) * q) return;
  const int i = int(idx / q), j = int(idx % q);
  Y[idx] = Z[int64_t(nlock + j) * ldz + nnow + i];
}

namespace {
struct HLWork {
  double *Y, *Y2, *G, *Rinv, *cholw, *Cs, *scr;
  int* status;
};
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
HLWork hl_carve(void* work, int m, int q) {
  char* c = static_cast<char*>(work);
  HLWork w;
  auto take = [&](size_t n) {
    double* r = reinterpret_cast<double*>(c);
    c += al256(n * sizeof(double));
    return r;
  };
  w.Y = take(size_t(m) * q);
  w.Y2 = take(size_t(m) * q);
  w.G = take(size_t(q) * q);
  w.Rinv = take(size_t(q) * q);
  w.cholw = take(size_t(q) * q + 2 * size_t(q));
  w.Cs = take(size_t(m) * q);
  w.scr = take(gram_scratch_elems(m, q, q, true));
  w.status = reinterpret_cast<int*>(c);
  return w;
}
}  // namespace

size_t hl_work_bytes(int s, int nnow, int nlock) {
  const size_t m = size_t(s - nnow), q = size_t(nnow - nlock);
  return 3 * al256(m * q * sizeof(double)) + 2 * al256(q * q * sizeof(double)) + al256((q * q + 2 * q) * sizeof(double)) +
         al256(gram_scratch_elems(int64_t(m), int(q), int(q), true) * sizeof(double)) + 256;
}

cudaError_t hl_trick(int s, int nnow, int nlock, const double* Z, int64_t ldz, double* CP, int64_t ldcp,
                     void* work, cudaStream_t st) {
  const int m = s - nnow, q = nnow - nlock;
  if (q <= 0) return cudaSuccess;
  if (m < q) return cudaErrorInvalidValue;
  HLWork w = hl_carve(work, m, q);
  hl_gather_kernel<<<(unsigned)cdiv(int64_t(m) * q, 256), 256, 0, st>>>(nnow, nlock, m, q, Z, ldz, w.Y);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  double* y = w.Y;
  double* y2 = w.Y2;
  for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
    Blk<double> Yb, Yo;
    Yb.add(y, q, q);
    Yo.add(y2, q, q);
    e = gram<Arith::F64>(m, Yb, Yb, true, w.G, q, w.scr, st);
    if (e == cudaSuccess) e = chol_rinv(q, m, w.G, q, w.Rinv, w.cholw, w.status, st, nullptr, 1.1102230246251565e-16);
    if (e == cudaSuccess) e = stage_coef<Arith::F64>(q, q, w.Rinv, q, w.Cs, q, 1.0, st);
    if (e == cudaSuccess) e = update<Arith::F64>(m, Yb, w.Cs, q, Yo, 0.0, st);
    std::swap(y, y2);
  }
  if (e != cudaSuccess) return e;
  // CP = Z(:, nnow:s) Q
  Blk<double> Zr, Cb;
  Zr.add(const_cast<double*>(Z) + nnow, ldz, m);
  Cb.add(CP, ldcp, q);
  e = stage_coef<Arith::F64>(m, q, y, q, w.Cs, q, 1.0, st);
  if (e == cudaSuccess) e = update<Arith::F64>(s, Zr, w.Cs, q, Cb, 0.0, st);
  return e;
}

}  // namespace eig
