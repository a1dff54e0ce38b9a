// Block products on the tensor cores: the Gram products G = U^T V and the
// block updates Y = U C + beta Y of the Rayleigh-Ritz, orthogonalisation and
// update steps of arXiv:2409.05572 (Algorithms 1-3), the two contractions
// that dominate every iteration.  This file cuts the operands into exact bf16
// slices (the scheme and the slice layout are described in tc.cuh) and
// dispatches the tcgen05 product kernel of k_tc5.cu.
//
//  Gram G = U^T V:   A = U^T, B = V^T, K = the n rows; chunks are 128 rows of
//                    one column (tc_slice_cols).
//  Update U C:       A = U, B = C^T, K = the s columns of U; chunks are 128
//                    columns of one row of U (tc_slice_rows) and 128 rows of one
//                    column of C (tc_slice_coef, from float64 C).
//
// Cutting.  Float64 values (7 slices) are cut from their bit patterns with
// integer operations only, so no FP64 instruction runs in an n-sized loop:
// with E the biased exponent of x and E_max that of the chunk's largest
// magnitude (e = E_max - 1022, max |x| < 2^e), the integer
//   F = x 2^(55 - e) = +- mantissa(x) 2^(E - E_max + 2)
// (right shifts round half away from zero) has |F| < 2^55 and its balanced
// base-256 digits are the slices.  Subnormal values count as zero; an
// infinite or NaN value makes its own slices NaN so that the product shows
// it.  Double-float values (6 slices) are cut in fp32: scaled by 2^(7 - e),
// the integer part of hi + lo is removed six times (rint, then TwoSum with
// the low part).  Chunks of a double-float operand whose maximum is below
// 2^-100 count as zero (their products are far below the rounding of any
// entry that matters; double-float itself has the float32 exponent range).
#include <cstring>
#include <type_traits>

#include "blocks.cuh"
#include "tc.cuh"

namespace eig {

using namespace tc;

namespace {

__device__ __forceinline__ float small_int_float(int d) {  // exact for |d| < 2^22
  return __int_as_float(0x4B400000 + d) - 12582912.0f;
}

// the NS prescaled slices s[q] = d_q 2^(-8 q) of one float64 bit pattern
// against a chunk whose largest biased exponent is emax (emax == 0: zero
// chunk).  Generic in NS: F = x 2^(8 NS - 1 - e), |F| < 2^(8 NS - 1).  The
// balanced base-256 digits of F are read off G = F + 0x80...80 (0x80 in each
// of the NS - 1 low bytes): low byte q of G is d + 128 for the balanced digit
// d at that position (the carries of the balanced representation are exactly
// those of the biased sum), and G >> 8 (NS - 1) is the top digit.
template <int NS>
__device__ __forceinline__ void cut_bits(unsigned long long bits, int emax, float* s) {
  static_assert(NS >= 2 && NS <= 7, "digit positions within 64 bits");
  // branch-free (selects only), so that the independent cuts of a thread
  // interleave
  const int E = int((bits >> 52) & 0x7FF);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - emax + 8 * NS - 54;      // <= 2
  const int ls = sh > 0 ? sh : 0;             // left shift
  const int rs = sh < 0 ? min(-sh, 63) : 0;   // right shift, rounding half away from zero
  const unsigned long long half = rs > 0 ? (1ull << max(rs - 1, 0)) : 0ull;
  unsigned long long u = ((m + half) >> rs) << ls;
  u = (E == 0 || emax == 0 || sh <= -60) ? 0ull : u;
  const long long F = (bits >> 63) ? -static_cast<long long>(u) : static_cast<long long>(u);
  constexpr unsigned long long BIAS = 0x8080808080808080ull >> (8 * (9 - NS));  // NS - 1 bytes of 0x80
  const unsigned long long G = static_cast<unsigned long long>(F) + BIAS;
  const uint32_t lo = static_cast<uint32_t>(G), hi = static_cast<uint32_t>(G >> 32);
#pragma unroll
  for (int q = NS - 1; q >= 1; --q) {
    const int pos = NS - 1 - q;  // byte position of digit q
    const uint32_t byte = pos < 4 ? (lo >> (8 * pos)) & 255u : (hi >> (8 * (pos - 4))) & 255u;
    // (2^23 + 2^22 + byte - 128) - (2^23 + 2^22) = d, exact; times 2^(-8 q)
    const float sc = __int_as_float((127 - 8 * q) << 23);
    s[q] = fmaf(__int_as_float(0x4B400000 - 128 + int(byte)), sc, -12582912.0f * sc);
  }
  const int top = static_cast<int>(static_cast<long long>(G) >> (8 * (NS - 1)));
  s[0] = small_int_float(top);
  if (E == 0x7FF) {  // infinity or NaN: poison the product
#pragma unroll
    for (int q = 0; q < NS; ++q) s[q] = __int_as_float(0x7fc00000);
  }
}

// Seven slices of two float64 values against a chunk with largest biased
// exponent emax, packed as bf16 pairs: word[q] holds slice q of the first
// value in its low half and of the second in its high half.  The same digits
// as cut_bits<7>, computed with 32-bit pieces: t = mantissa 2^2 is shifted
// right by emax - E >= 0 with rounding half away from zero (on the
// magnitude), F = +- that, G = F + 0x808080808080.  A digit's float is
// assembled from its byte with one byte permute (0x4B4000bb = 1.5 2^23 + bb),
// then scaled and offset by one exact FMA; the bf16 halves are the high 16
// bits of those exactly representable floats.  Infinite and NaN values are
// handled per chunk by the caller.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
__device__ __forceinline__ unsigned long long f64_biased_digits(unsigned long long bits, int emax) {
  const uint32_t hi = static_cast<uint32_t>(bits >> 32);
  const int E = int((hi >> 20) & 0x7FFu);
  const int r2 = emax - E;                               // >= 0 inside the chunk
  const unsigned long long t = ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2;
  const int r1 = min(max(r2 - 1, 0), 63);
  const unsigned long long v = t >> r1;
  unsigned long long u = r2 > 0 ? (v + 1ull) >> 1 : v;  // |x| 2^(E - emax + 2 + 52 - 52) rounded
  u = E == 0 ? 0ull : u;                                 // zero or subnormal
  const unsigned long long F = (hi >> 31) ? 0ull - u : u;
  return F + 0x808080808080ull;
}
__device__ __forceinline__ void cut2_f64(unsigned long long b0, unsigned long long b1, int emax, uint32_t* word) {
  const unsigned long long G0 = f64_biased_digits(b0, emax), G1 = f64_biased_digits(b1, emax);
  const uint32_t l0 = static_cast<uint32_t>(G0), h0 = static_cast<uint32_t>(G0 >> 32);
  const uint32_t l1 = static_cast<uint32_t>(G1), h1 = static_cast<uint32_t>(G1 >> 32);
  // digit q = 1 .. 6 sits in byte 6 - q of G: bytes 0..3 in the low word
#pragma unroll
  for (int q = 1; q < 7; ++q) {
    const int pos = 6 - q;
    const uint32_t sel = 0x7650u | uint32_t(pos & 3);
    const float c1 = __int_as_float((127 - 8 * q) << 23);  // 2^(-8 q)
    const float c2 = -12583040.0f * c1;                     // -(1.5 2^23 + 128) 2^(-8 q)
    const float f0 = __int_as_float(int(__byte_perm(pos < 4 ? l0 : h0, 0x4B400000u, sel)));
    const float f1 = __int_as_float(int(__byte_perm(pos < 4 ? l1 : h1, 0x4B400000u, sel)));
    word[q] = bf16_pair(fmaf(f0, c1, c2), fmaf(f1, c1, c2));
  }
  const int t0 = int(h0) >> 16, t1 = int(h1) >> 16;      // top digits, |d| <= 128
  word[0] = bf16_pair(small_int_float(t0), small_int_float(t1));
}

// the six prescaled slices of one double-float value times `scale` (a power
// of two): rint of the scaled value, the remainder (exact by Sterbenz)
// TwoSum-ed with the low part, times 256, six times
__device__ __forceinline__ void cut_dd(float hv, float lv, float scale, float* s) {
  hv *= scale;
  lv *= scale;
#pragma unroll
  for (int q = 0; q < NS_DF; ++q) {
    const float r = rintf(hv);
    s[q] = r * pow2(-8 * q);
    float nh, nl;
    two_sum(hv - r, lv, nh, nl);
    hv = nh * 256.f;
    lv = nl * 256.f;
  }
}

__device__ __forceinline__ int chunk_exp_dd(float mx) {
  int e = ZERO_EXP;
  if (mx >= 0x1p-100f) frexpf(mx, &e);  // 2^(e-1) <= mx < 2^e
  return e;
}

// the 16 values v[0..15][q] of one row, K indices 0 .. 15 of one block ->
// two 16-byte core-matrix rows
template <int NS>
__device__ __forceinline__ void store16(__nv_bfloat16* blk, int64_t r, const float (*v)[NS], int q) {
  uint32_t p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i][q], v[2 * i + 1][q]);
    p[i] = *reinterpret_cast<const uint32_t*>(&b);
  }
  *reinterpret_cast<uint4*>(blk + in_block(r, 0)) = make_uint4(p[0], p[1], p[2], p[3]);
  *reinterpret_cast<uint4*>(blk + in_block(r, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
}

template <typename T>
__device__ __forceinline__ void col_lookup(const Blk<T>& U, int c, const T*& p, int64_t& ld) {
  T* base;
  int s0;
  U.seg(c, base, ld, s0);
  p = base + (c - s0);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int nbytes) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_s() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_s() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// per-format pieces of the slicers: magnitude key of a raw 8-byte element
// (monotone in |x|), chunk exponent of the largest key, and the cut
template <typename T> struct SliceFmt;
template <> struct SliceFmt<dd> {
  static constexpr int NS = NS_DF;
  static __device__ __forceinline__ unsigned long long key(unsigned long long raw) {
    return __float_as_uint(fabsf(__uint_as_float(static_cast<uint32_t>(raw))));
  }
  static __device__ __forceinline__ int exp_of(unsigned long long k) {
    return chunk_exp_dd(__uint_as_float(static_cast<uint32_t>(k)));
  }
  // per-chunk cut parameter: the scale 2^(7 - e)
  using Prep = float;
  static __device__ __forceinline__ float prep(int e) { return e == ZERO_EXP ? 0.f : ldexpf(1.0f, 7 - e); }
  static __device__ __forceinline__ void cut(unsigned long long raw, float scale, float* s) {
    cut_dd(__uint_as_float(static_cast<uint32_t>(raw)), __uint_as_float(static_cast<uint32_t>(raw >> 32)), scale, s);
  }
  static __device__ __forceinline__ void cut2(unsigned long long r0, unsigned long long r1, float scale,
                                              uint32_t* word) {
    float s0[NS], s1[NS];
    cut(r0, scale, s0);
    cut(r1, scale, s1);
#pragma unroll
    for (int q = 0; q < NS; ++q) word[q] = bf16_pair(s0[q], s1[q]);
  }
  static __device__ __forceinline__ bool poisoned(float) { return false; }
};
template <> struct SliceFmt<double> {
  static constexpr int NS = NS_F64;
  static __device__ __forceinline__ unsigned long long key(unsigned long long raw) {
    return raw & 0x7FFFFFFFFFFFFFFFull;
  }
  // stored exponent e = E_max - 1022; biased E_max 0 (zero or subnormal) is a
  // zero chunk
  static __device__ __forceinline__ int exp_of(unsigned long long k) {
    const int E = int(k >> 52);
    return E == 0 ? ZERO_EXP : E - 1022;
  }
  // per-chunk cut parameter: the biased exponent E_max (0: zero chunk)
  using Prep = int;
  static __device__ __forceinline__ int prep(int e) { return e == ZERO_EXP ? 0 : e + 1022; }
  static __device__ __forceinline__ void cut(unsigned long long raw, int emax, float* s) {
    cut_bits<NS_F64>(raw, emax, s);
  }
  static __device__ __forceinline__ void cut2(unsigned long long r0, unsigned long long r1, int emax,
                                              uint32_t* word) {
    cut2_f64(r0, r1, emax, word);
  }
  // a chunk holding an infinity or a NaN (largest exponent field all ones):
  // its slices are NaN so that the products show it
  static __device__ __forceinline__ bool poisoned(int emax) { return emax == 0x7FF; }
};

// Slicer squares: one 128-index chunk of K x 32 operand rows, 256 threads,
// two shared-memory buffers of 128 x 33 (COLS) or 32 x 129 (ROWS) 8-byte
// elements.
constexpr int SQ_K = CH;   // 128
constexpr int SQ_M = 32;
constexpr int SL_P_COLS = SQ_M + 1, SL_P_ROWS = SQ_K + 1;
constexpr int SL_TILE = SQ_K * SQ_M + 128;  // elements per buffer (either pitch fits)
constexpr size_t SL_SHM = size_t(2) * SL_TILE * sizeof(unsigned long long);

// Both slicers: persistent CTAs walk the squares (a, b) of U, item = a nb + b;
// the next square's 8-byte loads are in flight (cp.async, two shared-memory
// buffers) while the current one is cut.
//  COLS (Gram operand): K = rows of U, operand rows = columns of U; square =
//       rows 128 a .. + 127 x columns 32 b .. + 31; one exponent per
//       (128-row chunk a, column).
//  ROWS (update operand): K = columns of U, operand rows = rows of U; square
//       = rows 32 a .. + 31 x columns 128 b .. + 127; one exponent per
//       (row, 128-column chunk b).
// The grids cover the padded operand rows, which get zero slices.
template <bool COLS, typename T>
__global__ void __launch_bounds__(256) tc_slice_kernel(int64_t n, Blk<T> U, Layout o, int64_t nb, int64_t items,
                                                       const int* gate) {
  using F = SliceFmt<T>;
  constexpr int NS = F::NS;
  if (gate && *gate == 0) return;
  constexpr int P = COLS ? SL_P_COLS : SL_P_ROWS;
  constexpr int ROWS_SQ = COLS ? SQ_K : SQ_M;  // rows of U in a square
  constexpr int COLS_SQ = COLS ? SQ_M : SQ_K;  // columns of U in a square
  constexpr int LC = COLS_SQ, LR = 256 / COLS_SQ;  // loader: LC columns x LR rows per step
  extern __shared__ __align__(16) unsigned long long sraw[];
  __shared__ unsigned long long pmax[8][32];
  __shared__ int sexp[32];
  const int t = threadIdx.x;
  const int w = U.width;
  int64_t item = blockIdx.x;
  if (item >= items) return;
  auto issue = [&](int64_t it, int buf) {
    const int64_t r0 = (it / nb) * ROWS_SQ;
    const int cb = int(it % nb) * COLS_SQ;
    const int lc = t % LC, lr = t / LC;
    const int c = cb + lc;
    const T* colp = nullptr;
    int64_t cld = 0;
    if (c < w) col_lookup(U, c, colp, cld);
    unsigned long long* dst = sraw + buf * SL_TILE;
#pragma unroll
    for (int i = 0; i < ROWS_SQ / LR; ++i) {
      const int rr = lr + LR * i;
      const int64_t r = r0 + rr;
      const bool ok = colp && r < n;
      cp_async8(dst + rr * P + lc, ok ? static_cast<const void*>(colp + r * cld) : static_cast<const void*>(U.ptr[0]),
                ok ? 8 : 0);
    }
    cp_async_commit_s();
  };
  issue(item, 0);
  int buf = 0;
  for (; item < items; item += gridDim.x) {
    const int64_t nxt = item + gridDim.x;
    if (nxt < items)
      issue(nxt, buf ^ 1);
    else
      cp_async_commit_s();
    cp_async_wait_s<1>();
    __syncthreads();
    const unsigned long long* sd = sraw + buf * SL_TILE;
    const int64_t a = item / nb, b = item % nb;
    if (COLS) {
      // column maxima over the 128 rows: 8 partial maxima per column
      const int lc = t & 31, lr = t >> 5;
      unsigned long long m = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) m = max(m, F::key(sd[(lr + 8 * i) * P + lc]));
      pmax[lr][lc] = m;
      __syncthreads();
      if (t < 32) {
        unsigned long long mm = pmax[0][t];
#pragma unroll
        for (int i = 1; i < 8; ++i) mm = max(mm, pmax[i][t]);
        const int e = F::exp_of(mm);
        sexp[t] = e;
        o.ex[a * o.Mp + b * SQ_M + t] = e;
      }
    } else {
      // row maxima over the 128 columns: 8 threads per row
      const int row = t >> 3, part = t & 7;
      unsigned long long m = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) m = max(m, F::key(sd[row * P + part + 8 * i]));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 4));
      if (part == 0) {
        const int e = F::exp_of(m);
        sexp[row] = e;
        o.ex[b * o.Mp + a * SQ_M + row] = e;
      }
    }
    __syncthreads();
    // thread -> (K block g of 16 indices, operand row idx of the square);
    // two halves of 8 K indices, each one 16-byte core-matrix row per slice
    const int g = t >> 5, idx = t & 31;
    const typename F::Prep pe = F::prep(sexp[idx]);
    const bool poison = F::poisoned(pe);
    const int64_t kb = (COLS ? a : b) * KBC + g;
    const int64_t orow = (COLS ? b : a) * SQ_M + idx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t w[4][NS];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 16 * g + 8 * h + 2 * i;
        F::cut2(COLS ? sd[k * P + idx] : sd[idx * P + k], COLS ? sd[(k + 1) * P + idx] : sd[idx * P + k + 1], pe,
                w[i]);
      }
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        uint4 v = make_uint4(w[0][q], w[1][q], w[2][q], w[3][q]);
        if (poison) v = make_uint4(0x7FC07FC0u, 0x7FC07FC0u, 0x7FC07FC0u, 0x7FC07FC0u);
        *reinterpret_cast<uint4*>(o.sl + o.block(q, kb) + in_block(orow, 8 * h)) = v;
      }
    }
    __syncthreads();  // the buffer is refilled by the next issue
    buf ^= 1;
  }
  cp_async_wait_s<0>();
}

// Update operand B from float64 C (s x c, ldc) times scale: K = rows of C,
// operand rows = columns of C.  Both formats cut the float64 bit patterns
// (NS = 6 with F = x 2^(47 - e)); for the double-float product, chunks below
// 2^-100 count as zero and the exponent must stay in the float range.
template <int NS>
__global__ void __launch_bounds__(256) tc_slice_coef_kernel(int s, int c, const double* __restrict__ C, int64_t ldc,
                                                            double scale, Layout o, const int* gate) {
  if (gate && *gate == 0) return;
  const int j0 = blockIdx.x * 32;
  const int kc = blockIdx.y;
  const int k00 = kc * CH;
  __shared__ unsigned long long sc[CH][33];
  __shared__ unsigned long long pmax[8][32];
  __shared__ int semax[32];
  const int t = threadIdx.x;
  {
    const int lj = t & 31, lk = t >> 5;
    const int j = j0 + lj;
    unsigned long long m = 0;
    for (int i = 0; i < CH / 8; ++i) {
      const int kk = lk + 8 * i;
      const int k = k00 + kk;
      const double x = (j < c && k < s) ? scale * C[int64_t(k) * ldc + j] : 0.0;
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
      sc[kk][lj] = b;
      m = max(m, b & 0x7FFFFFFFFFFFFFFFull);
    }
    pmax[lk][lj] = m;
  }
  __syncthreads();
  if (t < 32) {
    unsigned long long mm = pmax[0][t];
    for (int i = 1; i < 8; ++i) mm = max(mm, pmax[i][t]);
    int E = int(mm >> 52);
    if (NS == NS_DF && E < 1023 - 100) E = 0;  // below 2^-100: zero chunk
    semax[t] = E;
    o.ex[int64_t(kc) * o.Mp + j0 + t] = E == 0 ? ZERO_EXP : E - 1022;
  }
  __syncthreads();
  const int g = t >> 5, col = t & 31;
  const int emax = semax[col];
  float v[16][NS];
#pragma unroll
  for (int i = 0; i < 16; ++i) cut_bits<NS>(sc[16 * g + i][col], emax, v[i]);
  const int64_t kb = int64_t(kc) * KBC + g;
#pragma unroll
  for (int q = 0; q < NS; ++q) store16<NS>(o.sl + o.block(q, kb), j0 + col, v, q);
}

template <typename T> constexpr int ns_of() { return std::is_same<T, dd>::value ? NS_DF : NS_F64; }

template <bool COLS, typename T>
cudaError_t slice_launch(int64_t n, const Blk<T>& U, const Layout& o, int64_t na, int64_t nb, cudaStream_t st,
                         const int* gate) {
  static thread_local int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev != dev) {
    e = cudaFuncSetAttribute(tc_slice_kernel<COLS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SL_SHM));
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(tc_slice_kernel<COLS, T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    done_dev = dev;
  }
  const int64_t items = na * nb;
  int64_t grid = int64_t(num_sms()) * 3;  // three 67 KB CTAs per SM
  if (grid > items) grid = items;
  tc_slice_kernel<COLS, T><<<(unsigned)grid, 256, SL_SHM, st>>>(n, U, o, nb, items, gate);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

size_t tc_slice_bytes(int ns, int64_t K, int64_t M) { return slice_bytes(ns, K, M); }

size_t gram_tc_scratch_elems(int ns, int64_t n, int a, int b, bool sym) {
  return size_t(tc5_gram_nsplit(ns, n, a, b, sym)) * size_t(a) * size_t(b);
}

template <typename T>
cudaError_t tc_slice_cols(int64_t n, const Blk<T>& U, void* buf, cudaStream_t st, const int* gate) {
  const int w = U.width;
  if (w <= 0 || n <= 0) return cudaSuccess;
  const Layout o = layout(buf, ns_of<T>(), n, w);
  // squares: 128-row chunks of U (K) x 32-column blocks (operand rows, padded)
  return slice_launch<true, T>(n, U, o, cdiv(n, CH), o.Mp / SQ_M, st, gate);
}

template <typename T>
cudaError_t tc_slice_rows(int64_t n, const Blk<T>& U, void* buf, cudaStream_t st, const int* gate) {
  const int w = U.width;
  if (w <= 0 || n <= 0) return cudaSuccess;
  const Layout o = layout(buf, ns_of<T>(), w, n);
  // squares: 32-row blocks of U (operand rows, padded) x 128-column chunks (K)
  return slice_launch<false, T>(n, U, o, o.Mp / SQ_M, cdiv(w, CH), st, gate);
}

template cudaError_t tc_slice_cols<dd>(int64_t, const Blk<dd>&, void*, cudaStream_t, const int*);
template cudaError_t tc_slice_cols<double>(int64_t, const Blk<double>&, void*, cudaStream_t, const int*);
template cudaError_t tc_slice_rows<dd>(int64_t, const Blk<dd>&, void*, cudaStream_t, const int*);
template cudaError_t tc_slice_rows<double>(int64_t, const Blk<double>&, void*, cudaStream_t, const int*);

cudaError_t tc_slice_coef(int ns, int s, int c, const double* C, int64_t ldc, double scale, void* buf,
                          cudaStream_t st, const int* gate) {
  if (s <= 0 || c <= 0) return cudaSuccess;
  const Layout o = layout(buf, ns, s, c);
  dim3 grid((unsigned)(o.Mp / 32), (unsigned)cdiv(s, CH));
  if (ns == NS_DF)
    tc_slice_coef_kernel<NS_DF><<<grid, 256, 0, st>>>(s, c, C, ldc, scale, o, gate);
  else
    tc_slice_coef_kernel<NS_F64><<<grid, 256, 0, st>>>(s, c, C, ldc, scale, o, gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gram_tc_product(int ns_slices, int64_t n, int a, int b, const void* slu, const void* slv, bool sym,
                            double* G, int64_t ldg, double* scratch, cudaStream_t st, const int* gate) {
  if (a <= 0 || b <= 0 || n <= 0) return cudaSuccess;
  const int ns = tc5_gram_nsplit(ns_slices, n, a, b, sym);
  cudaError_t e = ns_slices == NS_DF ? tc5_gram<NS_DF>(n, a, b, slu, slv, sym, scratch, ns, st, gate)
                                     : tc5_gram<NS_F64>(n, a, b, slu, slv, sym, scratch, ns, st, gate);
  if (e != cudaSuccess) return e;
  return gram_reduce(a, b, ns, sym, scratch, G, ldg, st, gate);
}

template <typename T>
cudaError_t update_tc_product(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<T>& Y,
                              double beta, cudaStream_t st, const int* gate) {
  if (n <= 0 || c <= 0) return cudaSuccess;
  return tc5_update<ns_of<T>(), T>(n, s, c, slu, slc, Y, beta, st, gate);
}
template cudaError_t update_tc_product<dd>(int64_t, int, int, const void*, const void*, const Blk<dd>&, double,
                                           cudaStream_t, const int*);
template cudaError_t update_tc_product<double>(int64_t, int, int, const void*, const void*, const Blk<double>&,
                                               double, cudaStream_t, const int*);

cudaError_t tc_wait_selftest(int ns_slices, int64_t n, int a, int b, const void* slu, const void* slv,
                             double* scratch, double wait_s, cudaStream_t st) {
  const uint64_t ns = wait_s <= 0 ? 1000000ull : uint64_t(wait_s * 1e9);
  return tc5_wait_selftest(ns_slices, n, a, b, slu, slv, scratch, ns, st);
}

}  // namespace eig
