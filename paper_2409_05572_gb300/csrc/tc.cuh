// Shared pieces of the tensor-core block products (k_tc.cu: slicing and
// dispatch; k_tc5.cu: the tcgen05 product kernel).
//
// Two operand formats, one exact scheme (a fixed-point form of Ozaki, Ogita,
// Oishi and Rump, Numer. Algorithms 59, 2012):
//   NS = 6  double-float operands (EIG_ARITH_DF64_TC): six slices, the 21
//           slice pairs of levels 0..5, double-float result;
//   NS = 7  float64 operands (EIG_ARITH_F64_TC): seven slices, the 28 slice
//           pairs of levels 0..6, float64 result.
// A value x of a chunk whose largest magnitude is below 2^e is written as
//   x 2^(7 - e) = d_0 + d_1 2^-8 + ... + d_{NS-1} 2^(-8 (NS-1)) + r,
// balanced base-256 digits |d_i| <= 128, and slice i stores d_i 2^(-8 i) in
// bf16 (exact: at most 8 significant bits, exponent >= -56).  A product of
// slices i and j is then d_i t_j 2^(-8 (i + j)): exact in fp32, and the
// products of one level l = i + j over one chunk of 128 contraction indices
// sum to an integer multiple of 2^(-8 l) below 2^24 2^(-8 l) (at most NS
// pairs x 128 indices x 2^14 < 2^24), so each level accumulates EXACTLY in
// its own fp32 accumulator whatever order the tensor core adds in.
//
// Slice buffer of an operand with contraction length K and M operand rows
// (M padded to Mp, a multiple of 128; K padded to whole 128-index chunks):
//   slices: [NS][nkb][Mp][16] bf16, nkb = 16-index K blocks.  Inside one
//           (slice, K block) the Mp x 16 values are stored as 8 x 8 core
//           matrices, rows of 16 bytes: element (r, k) at
//           (r / 8) * 128 + (k / 8) * 64 + (r % 8) * 8 + k % 8,
//           so any 8-row-aligned run of rows is one contiguous range (one bulk
//           copy) whose shared-memory image is the no-swizzle K-major layout
//           of tcgen05.mma (core matrices 128 bytes apart along K, 256 bytes
//           apart along M).
//   exponents: [nkc][Mp] int after the slices, nkc = 128-index chunks; a
//           chunk whose values are all zero (or below the format's range)
//           has exponent ZERO_EXP and zero slices.
// Padding rows and K indices hold zeros.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace eig {
namespace tc {

constexpr int KB = 16;      // K indices per block (one tcgen05.mma K step)
constexpr int CH = 128;     // K indices per chunk (one exponent, one exact-level flush)
constexpr int KBC = CH / KB;
constexpr int MPAD = 128;   // operand rows are padded to this
constexpr int ZERO_EXP = -30000;
constexpr int NS_DF = 6;    // slices of a double-float value
constexpr int NS_F64 = 7;   // slices of a float64 value

__host__ __device__ inline int64_t nkb_of(int64_t K) { return ((K + CH - 1) / CH) * KBC; }
__host__ __device__ inline int64_t mpad_of(int64_t M) { return ((M + MPAD - 1) / MPAD) * MPAD; }

// element offset of (row r, K index k within the block) inside one block
__host__ __device__ inline int64_t in_block(int64_t r, int k) {
  return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

struct Layout {
  __nv_bfloat16* sl;
  int* ex;
  int64_t nkb, M, Mp;
  int ns;
  __host__ __device__ int64_t block(int q, int64_t kb) const { return (int64_t(q) * nkb + kb) * Mp * KB; }
};

inline Layout layout(const void* buf, int ns, int64_t K, int64_t M) {
  Layout o;
  o.ns = ns;
  o.nkb = nkb_of(K);
  o.M = M;
  o.Mp = mpad_of(M);
  o.sl = static_cast<__nv_bfloat16*>(const_cast<void*>(buf));
  o.ex = reinterpret_cast<int*>(o.sl + size_t(ns) * size_t(o.nkb) * size_t(o.Mp) * KB);
  return o;
}

// bytes of one slice buffer
inline size_t slice_bytes(int ns, int64_t K, int64_t M) {
  const size_t mp = size_t(mpad_of(M));
  return sizeof(__nv_bfloat16) * size_t(ns) * size_t(nkb_of(K)) * mp * KB +
         sizeof(int) * size_t((K + CH - 1) / CH) * mp;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// 2^k by its bit pattern; k > 127 gives +inf, k < -126 gives 0
__device__ __forceinline__ float pow2(int k) {
  return k > 127 ? __int_as_float(0x7f800000) : (k < -126 ? 0.f : __int_as_float((k + 127) << 23));
}

// master (double-float) += (hi + lo) * sc, sc a power of two or zero
__device__ __forceinline__ void add_scaled(dd& m, float hi, float lo, float sc) {
  float s, e;
  two_sum(m.hi, hi * sc, s, e);
  e += m.lo + lo * sc;
  m.hi = s + e;
  m.lo = e - (m.hi - s);
}

// Six prescaled level sums (a_l = L_l 2^(-8 l), exact) -> (hi, lo): the two
// leading terms error-free (TwoSum), the rest into lo.  |a_0| <= 2^21, so
// the roundings of lo stay below about 2^-23, 2^-44 of the largest chunk sum.
__device__ __forceinline__ void combine6(const float* a, float& hi, float& lo) {
  float h, e1, e2;
  two_sum(a[0], a[1], h, e1);
  two_sum(h, a[2], hi, e2);
  lo = e1 + e2;
  lo += a[3];
  lo += a[4];
  lo += a[5];
}

// Seven prescaled level sums -> hi + lo + small with hi + lo EXACT for
// levels 0..3 and small = a_4 + a_5 + a_6 (two roundings below 2^-33, i.e.
// 2^-54 of the largest chunk sum 2^21).  Levels 1..3 are split at multiples
// of 1/2 by the magic constant 1.5 * 2^22 (exact for |a| < 2^21; the level
// sums are below 2^14, 2^6.6 and 1): hi = a_0 + the three 1/2-multiples is a
// multiple of 1/2 below 2^22 (exact), lo = the three remainders, multiples
// of 2^-24 of magnitude <= 3/4 (exact).
__device__ __forceinline__ void combine7(const float* a, float& hi, float& lo, float& small) {
  constexpr float MAGIC = 6291456.0f;  // 1.5 * 2^22: its ulp is 1/2
  float h1 = __fadd_rn(a[1], MAGIC);
  h1 = __fsub_rn(h1, MAGIC);
  float h2 = __fadd_rn(a[2], MAGIC);
  h2 = __fsub_rn(h2, MAGIC);
  float h3 = __fadd_rn(a[3], MAGIC);
  h3 = __fsub_rn(h3, MAGIC);
  hi = __fadd_rn(__fadd_rn(a[0], h1), __fadd_rn(h2, h3));
  lo = __fadd_rn(__fadd_rn(__fsub_rn(a[1], h1), __fsub_rn(a[2], h2)), __fsub_rn(a[3], h3));
  small = __fadd_rn(__fadd_rn(a[4], a[5]), a[6]);
}

// one operand of a product kernel
struct Opnd {
  const __nv_bfloat16* sl;
  const int* ex;
  int64_t M, Mp;
};
inline Opnd opnd(const void* buf, int ns, int64_t K, int64_t M) {
  Layout l = layout(buf, ns, K, M);
  return Opnd{l.sl, l.ex, l.M, l.Mp};
}

struct GramOut {
  double* part;  // [split][M_A][M_B] float64 partial tiles
  bool sym;
};

// Y = P + beta Y of an update; T = dd (NS = 6) or double (NS = 7)
template <typename T>
struct UpdOut {
  Blk<T> Y;
  double beta;
  bool has_beta;
};

// the tcgen05 product kernels (k_tc5.cu)
template <int NS>
cudaError_t tc5_gram(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* scratch, int ns,
                     cudaStream_t st, const int* gate);
template <int NS, typename T>
cudaError_t tc5_update(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<T>& Y, double beta,
                       cudaStream_t st, const int* gate);
// split-K count of tc5_gram for NS = ns_slices
int tc5_gram_nsplit(int ns_slices, int64_t n, int a, int b, bool sym);
// one Gram product whose producer withholds its first stage (bounded-wait
// self-test; the kernel ends early after wait_ns with the error word set)
cudaError_t tc5_wait_selftest(int ns_slices, int64_t n, int a, int b, const void* slu, const void* slv,
                              double* scratch, uint64_t wait_ns, cudaStream_t st);
// 1 if a bounded wait of the tcgen05 kernels expired since the last call
// (then cleared), 0 if not, -1 if the flag could not be read
int tc5_take_error();

}  // namespace tc
}  // namespace eig
