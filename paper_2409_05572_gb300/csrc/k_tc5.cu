// tcgen05 product kernel of the sliced block products: the Gram products
// G = U^T V and the block updates Y = U C + beta Y of the Rayleigh-Ritz,
// orthogonalisation and update steps (Algorithms 1-3 of arXiv:2409.05572).
// The exact slicing and the slice layout are described in tc.cuh; NS = 6
// slices for double-float operands, NS = 7 for float64 operands.
//
// Output tiles are 128 x BN.  BN = 32: two sets of NS level accumulators
// (NS x 32 TMEM columns each) alternate by chunk, so the flush of one chunk
// runs while the MMAs of the next fill the other set.  BN = 64: one set of
// NS x 64 columns; the MMAs of the next chunk wait until the flush warps have
// read the levels.
//
// One CTA per SM, 320 threads in three roles:
//   warp 0, one thread   producer: per 16-index K block, two tensor copies
//                        (cp.async.bulk.tensor, the TMA engine; one 4-D box
//                        of all NS slices each) of the A tile (128 rows, 4 KB
//                        per slice) and the B tile (BN rows) into a ring of
//                        stages; each stage completes an mbarrier by
//                        transaction count.  (One copy per slice was measured
//                        to cap the copy rate at about 55 GB/s per SM: the
//                        copy engine spends a fixed time per request.)
//   warp 1, one thread   MMA issuer: per K block, all slice pairs (i, j) with
//                        i + j < NS as tcgen05.mma (M = 128, N = BN .. 256,
//                        K = 16, bf16 in, fp32 out) into the TMEM accumulator
//                        of level i + j; tcgen05.commit frees the stage and,
//                        after the 8 K blocks of a 128-index chunk, hands the
//                        exact level sums to the flush warps.
//   warps 2..9           flush: each warp owns the 32 TMEM lanes (tile rows)
//                        of its lane quarter and half of the BN columns; per
//                        chunk it reads the NS levels (tcgen05.ld), releases
//                        the set to the issuer, combines the levels, scales
//                        by the chunk exponents and adds to an accumulator in
//                        registers (double-float for NS = 6, triple-float for
//                        NS = 7); at the end of a tile it writes the float64
//                        split-K partial (Gram) or Y (update).
// Shared-memory operands use the no-swizzle K-major canonical layout: 8 x 16
// byte core matrices, 128 bytes apart along K (leading byte offset) and 256
// bytes apart along M/N (stride byte offset).
//
// Scales.  NS = 6: the chunk value is multiplied by 2^(e_a - 7) 2^(e_b - 7)
// in fp32 (double-float has the float32 exponent range).  NS = 7: float64
// exponents do not fit a float, so each flush thread takes reference
// exponents r_a (its row) and r_b (each column) as the largest chunk
// exponents of the tile's K range, scales a chunk by 2^(e_a - r_a) 2^(e_b - r_b)
// <= 1 in fp32 (contributions below 2^-126 of the largest chunk drop out) and
// multiplies the float64 result by 2^(r_a + r_b - 14) at the end.
//
// Accuracy (NS = 7).  Per chunk, the seven level sums are combined into
// hi + lo (exact) + small (error at most 2^-54 of the largest possible chunk
// sum; tc.cuh, combine7); the dropped levels 7..12 and the residual of the
// seven-digit representation add at most about 8 * 2^-56 of max|a| max|b|
// per index.  The triple-float accumulator (m0, m1, m2) takes hi and lo by
// error-free TwoSums and rounds only in m2, whose magnitude stays below
// about 2^-29 of the sum, so over K = 128 m indices the error is at most
// about 2^-52 sum_chunks 128 M_a M_b + m 2^-53 sum_chunks |c_k| -- within the
// float64 dot-product bound gamma_K sum |a b| with the chunk maxima in place
// of the elements.
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises the
// abort flag, records the expiry in the device error word, lets the other
// roles leave their loops, waits (bounded) for its own copies and MMAs and
// frees TMEM before returning.  The self-test entry point withholds the
// copies of one stage so that a wait runs out on purpose.
#include <cuda.h>

#include <cstdint>
#include <mutex>
#include <type_traits>

#include "blocks.cuh"
#include "tc.cuh"

namespace eig {
namespace tc {

__device__ int g_tc5_error = 0;  // set when a bounded wait expired

namespace {

constexpr int BM = 128;                        // A rows per tile (MMA M)
constexpr uint32_t A_SLICE = BM * KB * 2;      // 4 KB
template <int NS, int BN> struct Cfg {
  static constexpr uint32_t B_SLICE = BN * KB * 2;
  static constexpr uint32_t STAGE = NS * (A_SLICE + B_SLICE);
  static constexpr int NST = int((210u * 1024u) / STAGE);   // stages in about 210 KB
  static constexpr size_t SMEM = size_t(NST) * STAGE + 1024;  // + alignment slack
  static constexpr int NSETS = BN == 32 ? 2 : 1;             // TMEM accumulator sets
  static constexpr uint32_t SET_COLS = uint32_t(NS * BN);
  static constexpr int GRP = 256 / BN;                       // B slices per MMA (N <= 256)
  static constexpr int COLS_T = BN / 2;                      // columns per flush thread
  // columns per TMEM read of a flush thread: 8 when the triple-float
  // accumulators of 32 columns leave no room for 16-column reads
  static constexpr int SUBW = (NS == 7 && BN == 64) ? 8 : 16;
  static_assert(NSETS * SET_COLS <= 512, "TMEM");
};
constexpr uint32_t TMEM_COLS = 512;
constexpr int FLUSH_WARPS = 8;
constexpr int THREADS = 32 * (2 + FLUSH_WARPS);
constexpr uint32_t LBO = 128, SBO = 256;
// instruction descriptor: D f32, A and B bf16, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}
constexpr uint64_t WAIT_NS = 2000000000ull;  // a wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the completion of the phase with the given parity; false
// when another role aborted or wait_ns passed (then this one aborts)
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t wait_ns) {
  const uint64_t t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (now_ns() - t0 > wait_ns) break;
    }
  }
  *abort = 1;
  atomicExch(&g_tc5_error, 1);
  return false;
}

// bounded wait that does not abort (draining at exit)
__device__ __noinline__ void mbar_drain(uint32_t bar, uint32_t parity, uint64_t wait_ns) {
  const uint64_t t0 = now_ns();
  while (!mbar_test(bar, parity))
    if (now_ns() - t0 > wait_ns) {
      atomicExch(&g_tc5_error, 1);
      return;
    }
}

// One tensor (TMA) copy of a box of the slice buffer described by tmap:
// coordinates (0, first 8-row group, K block, first slice); the box is all
// NS slices of a 16-index K block of BM (A) or BN (B) operand rows, landing
// in shared memory as [slice][8-row group][8 x 16 core-matrix pair], i.e.
// slice q of the tile at q * (rows * 32) bytes.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* tmap, int rowgroup, int kb, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(rowgroup), "r"(kb), "r"(0), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((LBO >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((SBO >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
  return d;
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

// All slice pairs (qi, qj), qi + qj < NS, of one 16-index K block, into the
// accumulator set at TMEM address tset.  The B slices lie in shared memory
// one after another at the same 256-byte row-group stride, so B slices
// qj .. qj + m - 1 form one operand of N = BN m rows; with D at column
// BN (qi + qj), the product of A slice qi with B slice qj lands in the
// columns of level qi + qj.  The qi = 0 products touch every level and come
// first: first = the first K block of a chunk (overwrite).
template <int NS, int BN>
__device__ __forceinline__ void mma_kstep(uint32_t tset, uint32_t sa, uint32_t sb, bool first) {
  using C = Cfg<NS, BN>;
#pragma unroll
  for (int qi = 0; qi < NS; ++qi)
#pragma unroll
    for (int qj = 0; qj < NS - qi; qj += C::GRP) {
      const int m = (NS - qi - qj) < C::GRP ? (NS - qi - qj) : C::GRP;
      mma(tset + uint32_t(BN * (qi + qj)), sdesc(sa + uint32_t(qi) * A_SLICE),
          sdesc(sb + uint32_t(qj) * C::B_SLICE), idesc(BN * m), (qi == 0 && first) ? 0u : 1u);
    }
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane of one level accumulator
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// 8 consecutive TMEM columns of this thread's lane of one level accumulator
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// the NS level accumulators (BN columns apart), SW = 16 or 8 columns each,
// one wait
template <int NS, int BN, int SW>
__device__ __forceinline__ void tmem_ld_levels(uint32_t taddr, float (*v)[SW]) {
  uint32_t r[NS][SW];
#pragma unroll
  for (int l = 0; l < NS; ++l) {
    if constexpr (SW == 16)
      tmem_ld16(taddr + uint32_t(BN * l), r[l]);
    else
      tmem_ld8(taddr + uint32_t(BN * l), r[l]);
  }
  tmem_wait_ld();
#pragma unroll
  for (int l = 0; l < NS; ++l)
#pragma unroll
    for (int i = 0; i < SW; ++i) v[l][i] = __uint_as_float(r[l][i]);
}

// accumulators: double-float (NS = 6) and triple-float (NS = 7)
struct tf {
  float m0, m1, m2;
};
__device__ __forceinline__ void acc_zero(dd& m) { m = {0.f, 0.f}; }
__device__ __forceinline__ void acc_zero(tf& m) { m = {0.f, 0.f, 0.f}; }

// chunk value of one element from its NS prescaled level sums, added with
// scale sc (a power of two or zero)
__device__ __forceinline__ void flush_one(dd& m, const float* a, float sc) {
  float hi, lo;
  combine6(a, hi, lo);
  add_scaled(m, hi, lo, sc);
}
// m0 + m1 + m2 += (hi + lo + small) sc: hi into m0 and lo into m1 by TwoSum
// (exact), the rounding errors and small into m2
__device__ __forceinline__ void flush_one(tf& m, const float* a, float sc) {
  float hi, lo, small;
  combine7(a, hi, lo, small);
  float s0, e0, s1, e1, s2, e2;
  two_sum(m.m0, hi * sc, s0, e0);
  two_sum(m.m1, lo * sc, s1, e1);
  two_sum(s1, e0, s2, e2);
  m.m0 = s0;
  m.m1 = s2;
  m.m2 += (e1 + e2) + small * sc;
}
__device__ __forceinline__ double acc_value(const dd& m) { return double(m.hi) + double(m.lo); }
__device__ __forceinline__ double acc_value(const tf& m) { return (double(m.m0) + double(m.m1)) + double(m.m2); }

// (m0 + m1 + m2) 2^e rounded once to float64, with integer operations only:
// GB300 runs float64 arithmetic at 1/64 of its float32 rate, and the five
// float64 operations per element of acc_value + ldexp made the epilogue of
// a 128 x 32 update tile (three 128-index chunks) slower than its MMAs.
// The three floats become 64-bit fixed-point integers in units of
// 2^(E0 - 187), E0 the biased exponent of m0 (m0's 24-bit mantissa shifted
// left by 37 bits, the others aligned to it; each tail loses less than one
// unit, at most 2^-60 |m0|), their sum is rounded to 53 bits (nearest even)
// and the float64 fields are assembled.  Zero, tiny or non-finite heads, a tail above the
// head and results outside the normal float64 range take the float64 path.
__device__ __forceinline__ long long tf_fixed(uint32_t b, int E0) {
  const int E = int((b >> 23) & 255u);
  if (E == 0) return 0;  // zero, or a subnormal below 2^-60 |m0| (E0 >= 64)
  const long long M = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = E - E0 + 37;
  const long long v = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> -sh) : 0ll);
  return (b >> 31) ? -v : v;
}
__device__ __forceinline__ double tf_value_scaled(const tf& m, int e) {
  const uint32_t b0 = __float_as_uint(m.m0), b1 = __float_as_uint(m.m1), b2 = __float_as_uint(m.m2);
  const int E0 = int((b0 >> 23) & 255u), E1 = int((b1 >> 23) & 255u), E2 = int((b2 >> 23) & 255u);
  if (E0 < 64 || E0 == 255 || E1 > E0 + 1 || E2 > E0 + 1 || E1 == 255 || E2 == 255)
    return ldexp(acc_value(m), e);
  // |terms| < 2^61, 2^62, 2^62: the sum cannot overflow
  const long long S = tf_fixed(b0, E0) + tf_fixed(b1, E0) + tf_fixed(b2, E0);
  if (S == 0) return 0.0;
  const unsigned long long a = S < 0 ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const int nb = 64 - __clzll((long long)a);
  unsigned long long mant;
  int sh = nb - 53;
  if (sh > 0) {
    mant = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++sh;
    }
  } else {
    mant = a << (-sh);
  }
  // value = mant 2^(sh + E0 - 187 + e), mant in [2^52, 2^53)
  const int biased = sh + E0 - 187 + e + 52 + 1023;
  if (biased < 1 || biased > 2046) return ldexp(acc_value(m), e);
  const unsigned long long bits =
      (S < 0 ? (1ull << 63) : 0ull) | ((unsigned long long)biased << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

template <int NS>
using AccT = std::conditional_t<NS == 6, dd, tf>;

// MODE 0: Gram (tile (blockIdx.y, blockIdx.x) of 128 x BN, K blocks
// [z * kb_per, (z + 1) * kb_per) of split z = blockIdx.z).
// MODE 1: update (persistent: tiles t = blockIdx.x + i * gridDim.x of the
// tiles_m x tiles_n output tiles, N fastest, all K blocks).
// withhold >= 0 (self-test only): the producer issues no copies for stage
// position withhold, so the issuer's wait for it runs out after wait_ns.
template <int MODE, int NS, int BN, typename T>
__global__ void __launch_bounds__(THREADS, 1) tc5_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, Opnd A, Opnd B,
                                                         int nkb, int kb_per, int tiles_n,
                                                         int nitems, GramOut go, UpdOut<T> uo, const int* gate,
                                                         int withhold, uint64_t wait_ns) {
  using C = Cfg<NS, BN>;
  constexpr int NST = C::NST;
  constexpr int NSETS = C::NSETS;
  constexpr int CT = C::COLS_T;
  constexpr uint32_t STAGE = C::STAGE;
  if (gate && *gate == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int item0, item_step, nitem_cta, kb0, nkb_item;
  if (MODE == 0) {
    if (go.sym && int(blockIdx.x) * BN + BN - 1 < int(blockIdx.y) * BM) return;  // below the diagonal
    item0 = int(blockIdx.y) * tiles_n + int(blockIdx.x);
    item_step = 1;
    nitem_cta = 1;
    kb0 = int(blockIdx.z) * kb_per;
    const int kb1 = min(kb0 + kb_per, nkb);
    nkb_item = kb1 > kb0 ? kb1 - kb0 : 0;
    if (nkb_item == 0) {  // empty split: a zero partial tile
      const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
      for (int i = threadIdx.x; i < BM * BN; i += THREADS) {
        const int64_t r = m0 + i / BN, c = n0 + i % BN;
        if (r < A.M && c < B.M) go.part[int64_t(blockIdx.z) * A.M * B.M + r * B.M + c] = 0.0;
      }
      return;
    }
  } else {
    item0 = blockIdx.x;
    item_step = gridDim.x;
    nitem_cta = item0 < nitems ? (nitems - 1 - item0) / item_step + 1 : 0;
    kb0 = 0;
    nkb_item = nkb;
    if (nitem_cta == 0 || nkb_item == 0) return;
  }
  const int nchunk = nkb_item / KBC;  // K blocks come in whole chunks
  const int kc0 = kb0 / KBC;

  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_full[NST], bar_empty[NST], bar_accf[NSETS], bar_acce[NSETS], bar_done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  volatile int* abort = &abort_s;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < NSETS; ++s) {
      mbar_init(smem_u32(&bar_accf[s]), 1);
      mbar_init(smem_u32(&bar_acce[s]), FLUSH_WARPS);
    }
    mbar_init(smem_u32(&bar_done), 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer ----------------
      int p = 0;
      for (int it = 0; it < nitem_cta && !*abort; ++it) {
        const int item = item0 + it * item_step;
        const int64_t m0 = int64_t(item / tiles_n) * BM, n0 = int64_t(item % tiles_n) * BN;
        for (int kbi = 0; kbi < nkb_item; ++kbi, ++p) {
          const int s = p % NST;
          if (p >= NST && !mbar_wait(smem_u32(&bar_empty[s]), uint32_t((p / NST - 1) & 1), abort, wait_ns)) break;
          if (p == withhold) continue;  // self-test: this stage never fills
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, STAGE);
          const int kb = kb0 + kbi;
          const uint32_t sa = base + uint32_t(s) * STAGE, sb = sa + NS * A_SLICE;
          tma_box(sa, &tmA, int(m0 / 8), kb, fb);
          tma_box(sb, &tmB, int(n0 / 8), kb, fb);
        }
      }
      // the last stages' copies have landed before the CTA may exit
      for (int pp = max(0, p - NST); pp < p; ++pp)
        if (pp != withhold) mbar_drain(smem_u32(&bar_full[pp % NST]), uint32_t((pp / NST) & 1), wait_ns);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int p = 0, c = 0;
      bool ok = true;
      for (int it = 0; it < nitem_cta && ok; ++it) {
        for (int ch = 0; ch < nchunk && ok; ++ch, ++c) {
          const int set = c % NSETS, use = c / NSETS;  // use-th time this set is filled
          if (use > 0 && !(ok = mbar_wait(smem_u32(&bar_acce[set]), uint32_t((use - 1) & 1), abort, wait_ns)))
            break;
          fence_after();
          const uint32_t tset = tmem + uint32_t(set) * C::SET_COLS;
          for (int h = 0; h < KBC; ++h, ++p) {
            const int s = p % NST;
            if (!(ok = mbar_wait(smem_u32(&bar_full[s]), uint32_t((p / NST) & 1), abort, wait_ns))) break;
            fence_after();
            const uint32_t sa = base + uint32_t(s) * STAGE, sb = sa + NS * A_SLICE;
            mma_kstep<NS, BN>(tset, sa, sb, h == 0);
            commit(smem_u32(&bar_empty[s]));
          }
          if (ok) commit(smem_u32(&bar_accf[set]));
        }
      }
      // every MMA has completed before TMEM is freed
      commit(smem_u32(&bar_done));
      mbar_drain(smem_u32(&bar_done), 0, wait_ns);
    }
    __syncwarp();
  } else {
    // ---------------- flush warps ----------------
    const int quarter = warp & 3;                    // TMEM lanes 32 quarter .. + 31
    const int half = (warp - 2) >> 2;                // columns CT half .. + CT - 1
    const int rloc = 32 * quarter + lane;            // tile row of this thread
    const uint32_t trow = tmem + (uint32_t(32 * quarter) << 16) + uint32_t(CT * half);
    int c = 0;
    bool ok = true;
    for (int it = 0; it < nitem_cta && ok; ++it) {
      const int item = item0 + it * item_step;
      const int64_t m0 = int64_t(item / tiles_n) * BM, n0 = int64_t(item % tiles_n) * BN;
      const int* exa = A.ex + m0 + rloc;
      const int* exb = B.ex + n0 + CT * half + (lane % CT);  // lane j < CT holds column j's exponents
      // reference exponents: 7 (double-float), or the largest chunk
      // exponents of this tile's K range (float64)
      int ra = 7, rb = 7;
      if constexpr (NS == 7) {
        ra = ZERO_EXP;
        rb = ZERO_EXP;
        for (int ch = 0; ch < nchunk; ++ch) {
          ra = max(ra, exa[int64_t(kc0 + ch) * A.Mp]);
          rb = max(rb, exb[int64_t(kc0 + ch) * B.Mp]);
        }
      }
      AccT<NS> master[CT];
#pragma unroll
      for (int j = 0; j < CT; ++j) acc_zero(master[j]);
      for (int ch = 0; ch < nchunk; ++ch, ++c) {
        const int set = c % NSETS, use = c / NSETS;
        const int64_t kc = kc0 + ch;
        const float fa = pow2(exa[kc * A.Mp] - ra);
        const float fbl = pow2(exb[kc * B.Mp] - rb);
        if (!(ok = mbar_wait(smem_u32(&bar_accf[set]), uint32_t(use & 1), abort, wait_ns))) break;
        fence_after();
#pragma unroll
        constexpr int SW = C::SUBW;
        for (int sub = 0; sub < CT / SW; ++sub) {
          float v[NS][SW];
          tmem_ld_levels<NS, BN, SW>(trow + uint32_t(set) * C::SET_COLS + uint32_t(SW * sub), v);
          if (sub == CT / SW - 1) {  // levels read: the issuer may refill this set
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acce[set]));
          }
#pragma unroll
          for (int j = 0; j < SW; ++j) {
            float a[NS];
#pragma unroll
            for (int l = 0; l < NS; ++l) a[l] = v[l][j];
            const float fb = __shfl_sync(0xffffffffu, fbl, SW * sub + j);
            flush_one(master[SW * sub + j], a, fa * fb);
          }
        }
      }
      if (!ok) break;
      const int64_t r = m0 + rloc;
      const int64_t c0 = n0 + CT * half;
      const bool live = r < A.M;
      if (MODE == 0) {
#pragma unroll
        for (int j = 0; j < CT; ++j) {
          // float64 operands: times 2^(r_a + r_b(column) - 14); every lane
          // takes part in the shuffle
          double v;
          if constexpr (NS == 7)
            v = tf_value_scaled(master[j], ra - 14 + __shfl_sync(0xffffffffu, rb, j));
          else
            v = acc_value(master[j]);
          const int64_t col = c0 + j;
          if (live && col < B.M) go.part[int64_t(blockIdx.z) * A.M * B.M + r * B.M + col] = v;
        }
      } else {
        // when the thread's CT columns are one contiguous run of one segment
        // of Y, 16-byte aligned, write them as 16-byte vectors
        bool fast = false;
        T* yrow = nullptr;
        if (live && c0 + CT <= B.M) {
          T* yp;
          int64_t yld;
          int ys0;
          uo.Y.seg(int(c0), yp, yld, ys0);
          yrow = yp + r * yld + (c0 - ys0);
          // the run stays inside the segment when the column after it
          // belongs to the same one (or it ends the block)
          T* yq;
          int64_t qld;
          int qs0;
          uo.Y.seg(int(c0 + CT - 1), yq, qld, qs0);
          fast = qs0 == ys0 && (reinterpret_cast<uintptr_t>(yrow) & 15) == 0;
        }
        if constexpr (NS == 6) {
          if (live) {
            const float bh = float(uo.beta);
            const dd beta{bh, float(uo.beta - double(bh))};
            if (fast) {
              float4* y4 = reinterpret_cast<float4*>(yrow);
#pragma unroll
              for (int j = 0; j < CT; j += 2) {
                dd v0 = master[j], v1 = master[j + 1];
                if (uo.has_beta) {
                  const float4 old = y4[j / 2];
                  dd_mac(v0, dd{old.x, old.y}, beta);
                  dd_mac(v1, dd{old.z, old.w}, beta);
                }
                dd_renorm(v0);
                dd_renorm(v1);
                y4[j / 2] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
              }
            } else {
#pragma unroll
              for (int j = 0; j < CT; ++j) {
                const int64_t col = c0 + j;
                if (col < B.M) {
                  T* yp = uo.Y.at(r, int(col));
                  dd v = master[j];
                  if (uo.has_beta) dd_mac(v, *yp, beta);
                  dd_renorm(v);
                  *yp = v;
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < CT; j += 2) {
            // every lane takes part in the shuffles of the column exponents
            const int s0 = ra - 14 + __shfl_sync(0xffffffffu, rb, j);
            const int s1 = ra - 14 + __shfl_sync(0xffffffffu, rb, j + 1);
            double v0 = tf_value_scaled(master[j], s0);
            double v1 = tf_value_scaled(master[j + 1], s1);
            if (fast) {
              double2* y2 = reinterpret_cast<double2*>(yrow) + j / 2;
              if (uo.has_beta) {
                const double2 old = *y2;
                v0 = fma(uo.beta, old.x, v0);
                v1 = fma(uo.beta, old.y, v1);
              }
              *y2 = make_double2(v0, v1);
            } else if (live) {
              if (c0 + j < B.M) {
                T* yp = uo.Y.at(r, int(c0 + j));
                *yp = uo.has_beta ? fma(uo.beta, *yp, v0) : v0;
              }
              if (c0 + j + 1 < B.M) {
                T* yp = uo.Y.at(r, int(c0 + j + 1));
                *yp = uo.has_beta ? fma(uo.beta, *yp, v1) : v1;
              }
            }
          }
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

template <int MODE, int NS, int BN, typename T>
cudaError_t set_smem5() {
  static thread_local int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev != dev) {
    e = cudaFuncSetAttribute(tc5_kernel<MODE, NS, BN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(Cfg<NS, BN>::SMEM));
    if (e != cudaSuccess) return e;
    done_dev = dev;
  }
  return cudaSuccess;
}

int live_tiles(int a, int b, bool sym, int bn) {
  const int ta = (a + BM - 1) / BM, tb = (b + bn - 1) / bn;
  if (!sym) return ta * tb;
  int t = 0;
  for (int i = 0; i < ta; ++i)
    for (int j = 0; j < tb; ++j)
      if (!(j * bn + bn - 1 < i * BM)) ++t;
  return t;
}

template <int NS>
using ElemT = std::conditional_t<NS == 6, dd, double>;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// The slice buffer of an operand (ns slices, contraction length K, M rows;
// layout in tc.cuh) as a 4-D bf16 tensor, innermost first: the 128 values of
// one 8-row group of a K block (256 contiguous bytes), the Mp / 8 row groups
// (256 bytes apart), the K blocks (Mp * 32 bytes apart) and the slices;
// boxes of box_rows operand rows, one K block and all slices.
cudaError_t slice_tmap(CUtensorMap* m, const void* buf, int ns, int64_t K, int64_t M, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const Layout l = layout(buf, ns, K, M);
  const cuuint64_t dims[4] = {128, cuuint64_t(l.Mp / 8), cuuint64_t(l.nkb), cuuint64_t(ns)};
  const cuuint64_t strides[3] = {256, cuuint64_t(l.Mp) * 32, cuuint64_t(l.nkb) * cuuint64_t(l.Mp) * 32};
  const cuuint32_t box[4] = {128, cuuint32_t(box_rows / 8), 1, cuuint32_t(ns)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(buf), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// tile width of each product (see the head of this file): 128 x 64 for the
// double-float products and the float64 Grams, 128 x 32 with two alternating
// TMEM sets for the float64 updates (measured at n = 2^21: the float64 Gram
// 384 x 384 takes 16.5 ms with 64-wide tiles against 19.8 ms, the update
// 384 -> 256 24.4 ms against 23.4 ms)
template <int MODE, int NS> constexpr int bn_of() { return (NS == 6 || MODE == 0) ? 64 : 32; }

template <int NS>
cudaError_t gram_launch(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* scratch, int ns,
                        cudaStream_t st, const int* gate, int withhold, uint64_t wait_ns) {
  using T = ElemT<NS>;
  constexpr int BN = bn_of<0, NS>();
  cudaError_t e = set_smem5<0, NS, BN, T>();
  if (e != cudaSuccess) return e;
  const int64_t nkb = nkb_of(n);
  const int64_t kb_per = cdiv(cdiv(n, CH), ns) * KBC;
  const int tm = (a + BM - 1) / BM, tn = (b + BN - 1) / BN;
  GramOut go{scratch, sym};
  UpdOut<T> uo{};
  CUtensorMap tma, tmb;
  if ((e = slice_tmap(&tma, slu, NS, n, a, BM)) != cudaSuccess) return e;
  if ((e = slice_tmap(&tmb, slv, NS, n, b, BN)) != cudaSuccess) return e;
  dim3 grid(tn, tm, ns);
  tc5_kernel<0, NS, BN, T><<<grid, THREADS, Cfg<NS, BN>::SMEM, st>>>(tma, tmb, opnd(slu, NS, n, a),
                                                                      opnd(slv, NS, n, b), int(nkb), int(kb_per), tn,
                                                                      tm * tn, go, uo, gate, withhold, wait_ns);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int tc5_gram_nsplit(int ns_slices, int64_t n, int a, int b, bool sym) {
  const int bn = ns_slices == 6 ? bn_of<0, 6>() : bn_of<0, 7>();
  int ns = num_sms() / std::max(1, live_tiles(a, b, sym, bn));  // one CTA per SM, one wave
  const int64_t nch = cdiv(n, CH);
  if (ns > nch) ns = int(nch);
  if (ns < 1) ns = 1;
  return ns;
}

template <int NS>
cudaError_t tc5_gram(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* scratch, int ns,
                     cudaStream_t st, const int* gate) {
  return gram_launch<NS>(n, a, b, slu, slv, sym, scratch, ns, st, gate, -1, WAIT_NS);
}

template <int NS, typename T>
cudaError_t tc5_update(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<T>& Y, double beta,
                       cudaStream_t st, const int* gate) {
  static_assert(std::is_same<T, ElemT<NS>>::value, "slice count and element type disagree");
  constexpr int BN = bn_of<1, NS>();
  cudaError_t e = set_smem5<1, NS, BN, T>();
  if (e != cudaSuccess) return e;
  const int64_t nkb = nkb_of(s);
  const int64_t tm = cdiv(n, BM);
  const int tn = (c + BN - 1) / BN;
  const int64_t items = tm * tn;
  int64_t grid = num_sms();
  if (grid > items) grid = items;
  GramOut go{};
  UpdOut<T> uo;
  uo.Y = Y;
  uo.beta = beta;
  uo.has_beta = beta != 0.0;
  CUtensorMap tma, tmb;
  if ((e = slice_tmap(&tma, slu, NS, s, n, BM)) != cudaSuccess) return e;
  if ((e = slice_tmap(&tmb, slc, NS, s, c, BN)) != cudaSuccess) return e;
  tc5_kernel<1, NS, BN, T><<<(unsigned)grid, THREADS, Cfg<NS, BN>::SMEM, st>>>(
      tma, tmb, opnd(slu, NS, s, n), opnd(slc, NS, s, c), int(nkb), int(nkb), tn, int(items), go, uo, gate, -1,
      WAIT_NS);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t tc5_gram<6>(int64_t, int, int, const void*, const void*, bool, double*, int, cudaStream_t,
                                 const int*);
template cudaError_t tc5_gram<7>(int64_t, int, int, const void*, const void*, bool, double*, int, cudaStream_t,
                                 const int*);
template cudaError_t tc5_update<6, dd>(int64_t, int, int, const void*, const void*, const Blk<dd>&, double,
                                       cudaStream_t, const int*);
template cudaError_t tc5_update<7, double>(int64_t, int, int, const void*, const void*, const Blk<double>&, double,
                                           cudaStream_t, const int*);

// Self-test of the bounded waits: one Gram product (K = n, a x b, slices
// already made) whose producer withholds the copies of its first stage, so
// the MMA issuer's wait for that stage runs out after wait_ns and the kernel
// ends early with the device error word set.
cudaError_t tc5_wait_selftest(int ns_slices, int64_t n, int a, int b, const void* slu, const void* slv,
                              double* scratch, uint64_t wait_ns, cudaStream_t st) {
  const int ns = tc5_gram_nsplit(ns_slices, n, a, b, false);
  if (ns_slices == 6) return gram_launch<6>(n, a, b, slu, slv, false, scratch, ns, st, nullptr, 0, wait_ns);
  return gram_launch<7>(n, a, b, slu, slv, false, scratch, ns, st, nullptr, 0, wait_ns);
}

// status of the bounded waits since the last call (0: none expired); resets it
int tc5_take_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc5_error, sizeof(int)) != cudaSuccess) return -1;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc5_error, &z, sizeof(int));
  }
  return v;
}

}  // namespace tc
}  // namespace eig
