// Internal (C++) interface of the n-sized block kernels: SpMM, Gram, block
// update, residual, conversions.  Explicitly instantiated in k_blocks.cu.
#pragma once
#include "common.cuh"

namespace eig {

template <Arith A>
struct Csr {
  int64_t n = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const typename Pol<A>::T* val = nullptr;
  // rows with more than heavy_min nonzeros (the nheavy row indices in
  // heavy, device memory) are split over the warps of one CTA each instead
  // of one lane group; heavy_min = 0: no split
  const int32_t* heavy = nullptr;
  int nheavy = 0;
  int heavy_min = 0;
};

// Y = alpha A V + beta V + gamma U (single-segment n x w views)
template <Arith A>
cudaError_t spmm(const Csr<A>& M, int w, const typename Pol<A>::T* V, int64_t ldv,
                 typename Pol<A>::T* Y, int64_t ldy, double alpha, double beta,
                 const typename Pol<A>::T* U, int64_t ldu, double gamma, cudaStream_t st);

// Scratch (float64 elements) that gram() needs for its split-K partial tiles.
size_t gram_scratch_elems(int64_t n, int a, int b, bool sym);

// G (a x b, float64, ldg) = U^T V; scratch from gram_scratch_elems().
template <Arith A>
cudaError_t gram(int64_t n, const Blk<typename Pol<A>::T>& U, const Blk<typename Pol<A>::T>& V,
                 bool sym, double* G, int64_t ldg, double* scratch, cudaStream_t st,
                 const int* gate = nullptr);

// gram() with the split-K count limited so the partial tiles fit in
// max_scratch_elems float64 elements; cudaErrorInvalidValue if even one
// split does not fit (a * b > max_scratch_elems).
template <Arith A>
cudaError_t gram_capped(int64_t n, const Blk<typename Pol<A>::T>& U, const Blk<typename Pol<A>::T>& V,
                        bool sym, double* G, int64_t ldg, double* scratch, size_t max_scratch_elems,
                        cudaStream_t st);

// G[i][j] = sum over z < nsplit of part[z][i][j] (a x b partial tiles) in
// that fixed order; sym: the lower triangle mirrors the upper one.
cudaError_t gram_reduce(int a, int b, int nsplit, bool sym, const double* part, double* G, int64_t ldg,
                        cudaStream_t st, const int* gate = nullptr);

// Tensor-core products (k_tc.cu, k_tc5.cu) of double-float blocks (6 exact
// bf16 slices) and float64 blocks (7 slices).  A slice buffer holds the
// slices of an operand with contraction length K and M operand rows:
// tc_slice_bytes(ns, K, M) bytes, 16-byte aligned.
//  - Gram G = U^T V (n x a, n x b): tc_slice_cols() of U and V (K = n,
//    M = width), gram_tc_product() with split-K partial tiles in scratch
//    (gram_tc_scratch_elems() float64 elements).
//  - Update Y = U (scale C) + beta Y (U: n x s, C: s x c float64): tc_slice_rows()
//    of U (K = s, M = n), tc_slice_coef() of C (K = s, M = c),
//    update_tc_product().  Y must not overlap U.
// T = dd (ns = 6) or double (ns = 7).
size_t tc_slice_bytes(int ns, int64_t K, int64_t M);
size_t gram_tc_scratch_elems(int ns, int64_t n, int a, int b, bool sym);
template <typename T>
cudaError_t tc_slice_cols(int64_t n, const Blk<T>& U, void* buf, cudaStream_t st, const int* gate = nullptr);
template <typename T>
cudaError_t tc_slice_rows(int64_t n, const Blk<T>& U, void* buf, cudaStream_t st, const int* gate = nullptr);
cudaError_t tc_slice_coef(int ns, int s, int c, const double* C, int64_t ldc, double scale, void* buf,
                          cudaStream_t st, const int* gate = nullptr);
cudaError_t gram_tc_product(int ns, int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* G,
                            int64_t ldg, double* scratch, cudaStream_t st, const int* gate = nullptr);
template <typename T>
cudaError_t update_tc_product(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<T>& Y,
                              double beta, cudaStream_t st, const int* gate = nullptr);
// Bounded-wait self-test: a Gram product (slices made) whose first stage is
// withheld, so a wait of the product kernel runs out after wait_s seconds.
cudaError_t tc_wait_selftest(int ns, int64_t n, int a, int b, const void* slu, const void* slv, double* scratch,
                             double wait_s, cudaStream_t st);

// Cs[i][j] (leading dimension ldo) = staged(scale * C[i][j]) for an s x c
// float64 matrix.
template <Arith A>
cudaError_t stage_coef(int s, int c, const double* C, int64_t ldc, typename Pol<A>::S* Cs,
                       int64_t ldo, double scale, cudaStream_t st, const int* gate = nullptr);

// Y = a U + b V elementwise (n x w views; Y may alias U or V).
template <Arith A>
cudaError_t axpby(int64_t n, int w, const typename Pol<A>::T* U, int64_t ldu, double a,
                  const typename Pol<A>::T* V, int64_t ldv, double b, typename Pol<A>::T* Y,
                  int64_t ldy, cudaStream_t st);

// dst = src over n rows (equal widths), skipped when *gate == 0.
template <typename T>
cudaError_t copy_blk(int64_t n, const Blk<T>& src, const Blk<T>& dst, cudaStream_t st,
                     const int* gate = nullptr);

// Y = U Cs + beta Y, Cs staged s x c (leading dimension c); Y must not
// overlap U.
template <Arith A>
cudaError_t update(int64_t n, const Blk<typename Pol<A>::T>& U, const typename Pol<A>::S* Cs,
                   int c, const Blk<typename Pol<A>::T>& Y, double beta, cudaStream_t st,
                   const int* gate = nullptr);

// Scratch (float64 elements) for residual(): 2 * blocks * w.
size_t residual_scratch_elems(int64_t n, int w);

// R = T (AX - X diag(lam)); xnorm2, rnorm2 (float64, device, length w).
template <Arith A>
cudaError_t residual(int64_t n, int w, const typename Pol<A>::T* X, int64_t ldx,
                     const typename Pol<A>::T* AX, int64_t ldax, const double* lam,
                     const typename Pol<A>::T* tdiag, typename Pol<A>::T* R, int64_t ldr,
                     double* xnorm2, double* rnorm2, double* scratch, cudaStream_t st);

// Elementwise format conversion between float64, float32 and double-float
// for a rows x cols block (row-major, own leading dimensions).
cudaError_t convert2d(int64_t rows, int64_t cols, const void* src, int64_t lds, int sdt, void* dst,
                      int64_t ldd, int ddt, cudaStream_t st);

// n x w Gaussian columns of the 'Random' expansion (Sec. 6.4) in element
// format dt (EIG_F64, EIG_DF64, EIG_F32): a counter-based draw, entry (i, j)
// a function of (seed, e, i, j) only (k_blocks.cu)
cudaError_t gauss_fill(int64_t n, int w, void* dst, int64_t ld, int dt, uint64_t seed, int e, cudaStream_t st);

}  // namespace eig
