// Shared pieces of the tensor-core products of double-float blocks (k_tc.cu:
// slicing and the mma.sync product; k_tc5.cu: the tcgen05 product).
//
// Slice buffer of an operand with contraction length K and M operand rows
// (M padded to Mp, a multiple of 128; K padded to whole 128-index chunks):
//   slices: [TC_S][nkb][Mp][32] bf16, nkb = 32-index K blocks.  Inside one
//           (slice, K block) the Mp x 32 values are stored as 8 x 8 core
//           matrices, rows of 16 bytes: element (r, k) at
//           (r / 8) * 256 + (k / 8) * 64 + (r % 8) * 8 + k % 8,
//           so any 8-row-aligned run of rows is one contiguous range (one bulk
//           copy) and its shared-memory image is the no-swizzle K-major layout
//           of tcgen05.mma (core matrices 128 bytes apart along K, 512 bytes
//           apart along M).
//   exponents: [nkc][Mp] int after the slices, nkc = 128-index chunks.
// Padding rows and K indices hold zeros.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace eig {
namespace tc {

constexpr int S = 6;        // slices per value
constexpr int KB = 32;      // K indices per block
constexpr int CH = 128;     // K indices per chunk (one exponent, one exact-level flush)
constexpr int KBC = CH / KB;
constexpr int MPAD = 128;   // operand rows are padded to this
constexpr int ZERO_EXP = -1000;

__host__ __device__ inline int64_t nkb_of(int64_t K) { return ((K + CH - 1) / CH) * KBC; }
__host__ __device__ inline int64_t mpad_of(int64_t M) { return ((M + MPAD - 1) / MPAD) * MPAD; }

// element offset of (row r, K index k within the block) inside one block
__host__ __device__ inline int64_t in_block(int64_t r, int k) {
  return (r >> 3) * 256 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

struct Layout {
  __nv_bfloat16* sl;
  int* ex;
  int64_t nkb, M, Mp;
  __host__ __device__ int64_t block(int q, int64_t kb) const { return (int64_t(q) * nkb + kb) * Mp * KB; }
};

inline Layout layout(const void* buf, int64_t K, int64_t M) {
  Layout o;
  o.nkb = nkb_of(K);
  o.M = M;
  o.Mp = mpad_of(M);
  o.sl = static_cast<__nv_bfloat16*>(const_cast<void*>(buf));
  o.ex = reinterpret_cast<int*>(o.sl + size_t(S) * size_t(o.nkb) * size_t(o.Mp) * KB);
  return o;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// (hi, lo) = sum_l a_l 2^(-8 l) for exact integer level sums |a_l| < 2^24:
// the two leading terms error-free (TwoSum), the rest into lo.  With
// |a_0| <= 2^21 (one product per K index), |lo| < 2^0 and the four roundings
// of lo stay below 2^-23, i.e. 2^-44 of the largest possible chunk sum.
__device__ __forceinline__ void combine_levels(float a0, float a1, float a2, float a3, float a4, float a5,
                                               float& hi, float& lo) {
  float h, e1, e2;
  two_sum(a0, a1 * 0x1p-8f, h, e1);
  two_sum(h, a2 * 0x1p-16f, hi, e2);
  lo = e1 + e2;
  lo = fmaf(a3, 0x1p-24f, lo);
  lo = fmaf(a4, 0x1p-32f, lo);
  lo = fmaf(a5, 0x1p-40f, lo);
}

// 2^k by its bit pattern; k > 127 (a float64 coefficient beyond the float
// range) gives +inf, k < -126 gives 0
__device__ __forceinline__ float pow2(int k) {
  return k > 127 ? __int_as_float(0x7f800000) : (k < -126 ? 0.f : __int_as_float((k + 127) << 23));
}

// master (double-float) += (hi, lo) * sc
__device__ __forceinline__ void add_scaled(dd& m, float hi, float lo, float sc) {
  float s, e;
  two_sum(m.hi, hi * sc, s, e);
  e += m.lo + lo * sc;
  m.hi = s + e;
  m.lo = e - (m.hi - s);
}

}  // namespace tc
}  // namespace eig

namespace eig {
namespace tc {

// one operand of a product kernel
struct Opnd {
  const __nv_bfloat16* sl;
  const int* ex;
  int64_t M, Mp;
};
inline Opnd opnd(const void* buf, int64_t K, int64_t M) {
  Layout l = layout(buf, K, M);
  return Opnd{l.sl, l.ex, l.M, l.Mp};
}

struct GramOut {
  double* part;  // [split][M_A][M_B] float64 partial tiles
  bool sym;
};

struct UpdOut {
  Blk<dd> Y;
  dd beta;
  bool has_beta;
};

// the tcgen05 product kernels (k_tc5.cu); same arguments as the host
// functions gram_tc_product / update_tc_product
cudaError_t tc5_gram(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* scratch, int ns,
                     cudaStream_t st, const int* gate);
cudaError_t tc5_update(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<dd>& Y, double beta,
                       cudaStream_t st, const int* gate);
// split-K count of tc5_gram (tile 128 x 64)
int tc5_gram_nsplit(int64_t n, int a, int b, bool sym);
// 1 if a bounded wait of the tcgen05 kernels expired since the last call
// (then cleared), 0 if not, -1 if the flag could not be read
int tc5_take_error();

}  // namespace tc
}  // namespace eig
