// Internal (C++) interface of the small dense float64 kernels (k_small.cu).
#pragma once
#include "common.cuh"

namespace eig {

// R^{-1} (w x w upper, leading dimension w) of the Cholesky factor of G;
// unit_round is the unit roundoff of the data G came from (it sets the shift);
// *status: 0 plain, 1 shifted (Fukaya et al. 2020), 2 broken down.  work:
// (w*w + 2w) doubles, used when the factor does not fit in shared memory.
cudaError_t chol_rinv(int w, int64_t nrows, const double* G, int64_t ldg, double* Rinv, double* work,
                      int* status, cudaStream_t st, const int* gate = nullptr,
                      double unit_round = 1.1102230246251565e-16);

// A = Z diag(lam) Z^T, lam ascending, Z float64 (leading dimension ldz):
// float32 Householder tridiagonalisation, bisection and inverse iteration,
// then Ogita-Aishima refinement in double-float and Jacobi on clusters
// (k_syev.cu).  work of syev_work_bytes(s) bytes; *status_dev: 0 ok, 3 a
// cluster of nearly equal eigenvalues is larger than the Jacobi stage takes.
size_t syev_work_bytes(int s);
cudaError_t syev(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                 int* status_dev, cudaStream_t st);
// The same decomposition in float64: Householder, multisection bisection,
// inverse iteration with Gram-Schmidt inside clusters and one float64
// Ogita-Aishima step (syev64, work of syev64_work_bytes(s) bytes), or the
// sequential implicit QL chain (syev_qr64, a slow comparison path, work of
// syev_qr64_work_bytes(s) bytes).
size_t syev_qr64_work_bytes(int s);
size_t syev64_work_bytes(int s);
cudaError_t syev64(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                   int* status_dev, cudaStream_t st);
cudaError_t syev_qr64(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* work,
                      int* status_dev, cudaStream_t st);

// improved Hetmaniuk-Lehoucq: CP = Z(:, nnow:s) Q, Q the orthonormal QR
// factor (shifted CholeskyQR3) of Z(nlock:nnow, nnow:s)^T; work of
// hl_work_bytes() bytes.
size_t hl_work_bytes(int s, int nnow, int nlock);
cudaError_t hl_trick(int s, int nnow, int nlock, const double* Z, int64_t ldz, double* CP, int64_t ldcp,
                     void* work, cudaStream_t st);

}  // namespace eig
