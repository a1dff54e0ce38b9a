// tcgen05 product kernel of the sliced double-float products (Gram G = U^T V
// and update Y = U C + beta Y of Algorithms 1-3 of arXiv:2409.05572; the
// exact slicing and its error bound are described in k_tc.cu, the slice
// layout in tc.cuh).
//
// One CTA per SM, 320 threads in three roles:
//   warp 0, one thread   producer: per 32-index K block, 6 + 6 bulk copies
//                        (cp.async.bulk, the TMA engine) of the A tile
//                        (128 rows, 8 KB per slice) and the B tile (64 rows,
//                        4 KB per slice) into a 3-stage ring; each stage
//                        completes an mbarrier by transaction count.
//   warp 1, one thread   MMA issuer: per K block and 16-index half, the 21
//                        slice pairs (i, j), i + j <= 5, as eight tcgen05.mma
//                        (M = 128, N = 64 .. 256, K = 16, bf16 in, fp32 out)
//                        into the TMEM accumulators of the levels i + j (6 x 64
//                        columns); tcgen05.commit frees the stage and, after
//                        the last K block of a 128-index chunk, hands the
//                        six exact level sums to the flush warps.
//   warps 2..9           flush: each warp owns the 32 TMEM lanes (tile rows)
//                        of its lane quarter and 32 of the 64 columns; per
//                        chunk it reads the six levels (tcgen05.ld), releases
//                        TMEM to the issuer, combines the levels into a
//                        double-float, scales by 2^(e_a - 7) 2^(e_b - 7) and
//                        adds to its registers; at the end of a tile it writes
//                        the float64 partial (Gram) or Y (update).
// Shared-memory operands use the no-swizzle K-major canonical layout: 8 x 16
// byte core matrices, 128 bytes apart along K (leading byte offset) and 512
// bytes apart along M/N (stride byte offset).
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises the
// abort flag, records the expiry in the device error word, lets the other
// roles leave their loops, waits (bounded) for its own copies and MMAs and
// frees TMEM before returning.
#include <cstdint>
#include <cstdlib>

#include "blocks.cuh"
#include "tc.cuh"

namespace eig {
namespace tc {

__device__ int g_tc5_error = 0;  // set when a bounded wait expired

namespace {

constexpr int BM = 128;                        // A rows per tile (MMA M)
constexpr int BN = 64;                         // B rows per tile (MMA N)
constexpr int NST = 3;                         // stages of one 32-index K block
constexpr uint32_t A_SLICE = BM * KB * 2;      // 8 KB
constexpr uint32_t B_SLICE = BN * KB * 2;      // 4 KB
constexpr uint32_t STAGE = S * (A_SLICE + B_SLICE);
constexpr uint32_t TMEM_COLS = 512;            // 6 levels x 64 columns used
constexpr int FLUSH_WARPS = 8;
constexpr int THREADS = 32 * (2 + FLUSH_WARPS);
constexpr size_t SMEM = size_t(NST) * STAGE + 1024;  // + alignment slack
constexpr uint32_t LBO = 128, SBO = 512;
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
// when another role aborted or WAIT_NS passed (then this one aborts)
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const uint64_t t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (now_ns() - t0 > WAIT_NS) break;
    }
  }
  *abort = 1;
  atomicExch(&g_tc5_error, 1);
  return false;
}

// bounded wait that does not abort (draining at exit)
__device__ __noinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  while (!mbar_test(bar, parity))
    if (now_ns() - t0 > WAIT_NS) {
      atomicExch(&g_tc5_error, 1);
      return;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
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

// All slice pairs (qi, qj), qi + qj <= 5, of one 16-index K step.  The B
// slices lie in shared memory one after another with the same 512-byte
// row-group stride, so B slices qj .. qj + m - 1 form one operand of
// N = 64 m rows; with D at TMEM column 64 qi, the product of A slice qi with
// B slice qj lands in the columns of level qi + qj.  Eight MMAs (N <= 256)
// cover the 21 pairs.  first: the first K step of a chunk (overwrite).
__device__ __forceinline__ void mma_kstep(uint32_t tmem, uint32_t sa, uint32_t sb, bool first) {
  const uint32_t acc = first ? 0u : 1u;
  // qi = 0: levels 0..3 and 4..5 (these two start every level of the chunk)
  mma(tmem + 0 * BN, sdesc(sa + 0 * A_SLICE), sdesc(sb + 0 * B_SLICE), idesc(4 * BN), acc);
  mma(tmem + 4 * BN, sdesc(sa + 0 * A_SLICE), sdesc(sb + 4 * B_SLICE), idesc(2 * BN), acc);
  // qi = 1: levels 1..4 and 5
  mma(tmem + 1 * BN, sdesc(sa + 1 * A_SLICE), sdesc(sb + 0 * B_SLICE), idesc(4 * BN), 1u);
  mma(tmem + 5 * BN, sdesc(sa + 1 * A_SLICE), sdesc(sb + 4 * B_SLICE), idesc(1 * BN), 1u);
  // qi = 2 .. 5: levels qi .. 5
  mma(tmem + 2 * BN, sdesc(sa + 2 * A_SLICE), sdesc(sb), idesc(4 * BN), 1u);
  mma(tmem + 3 * BN, sdesc(sa + 3 * A_SLICE), sdesc(sb), idesc(3 * BN), 1u);
  mma(tmem + 4 * BN, sdesc(sa + 4 * A_SLICE), sdesc(sb), idesc(2 * BN), 1u);
  mma(tmem + 5 * BN, sdesc(sa + 5 * A_SLICE), sdesc(sb), idesc(1 * BN), 1u);
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane in each of the six
// level accumulators (64 columns apart), one wait for all six loads
__device__ __forceinline__ void tmem_ld_levels(uint32_t taddr, float (*v)[16]) {
  uint32_t r[96];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%96];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%97];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%98];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%99];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79}, [%100];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95}, [%101];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79]), "=r"(r[80]), "=r"(r[81]), "=r"(r[82]), "=r"(r[83]), "=r"(r[84]), "=r"(r[85]), "=r"(r[86]), "=r"(r[87]), "=r"(r[88]), "=r"(r[89]), "=r"(r[90]), "=r"(r[91]), "=r"(r[92]), "=r"(r[93]), "=r"(r[94]), "=r"(r[95])
      : "r"(taddr), "r"(taddr + 64u), "r"(taddr + 128u), "r"(taddr + 192u), "r"(taddr + 256u), "r"(taddr + 320u)
      : "memory");
#pragma unroll
  for (int l = 0; l < 6; ++l)
#pragma unroll
    for (int i = 0; i < 16; ++i) v[l][i] = __uint_as_float(r[16 * l + i]);
}

// MODE 0: Gram (tile (blockIdx.y, blockIdx.x) of 128 x 64, K blocks
// [z * kb_per, (z + 1) * kb_per) of split z = blockIdx.z).
// MODE 1: update (persistent: tiles t = blockIdx.x + i * gridDim.x of the
// tiles_m x tiles_n output tiles, N fastest, all K blocks).
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) tc5_kernel(Opnd A, Opnd B, int nkb, int kb_per, int tiles_n,
                                                         int nitems, GramOut go, UpdOut uo, const int* gate) {
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

  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_full[NST], bar_empty[NST], bar_accf, bar_acce, bar_done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  volatile int* abort = &abort_s;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_accf), 1);
    mbar_init(smem_u32(&bar_acce), FLUSH_WARPS);
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
          if (p >= NST && !mbar_wait(smem_u32(&bar_empty[s]), uint32_t((p / NST - 1) & 1), abort)) break;
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, STAGE);
          const int64_t kb = kb0 + kbi;
          const uint32_t sa = base + uint32_t(s) * STAGE, sb = sa + S * A_SLICE;
#pragma unroll 1
          for (int q = 0; q < S; ++q) {
            bulk_g2s(sa + q * A_SLICE, A.sl + (int64_t(q) * nkb + kb) * A.Mp * KB + m0 * KB, A_SLICE, fb);
            bulk_g2s(sb + q * B_SLICE, B.sl + (int64_t(q) * nkb + kb) * B.Mp * KB + n0 * KB, B_SLICE, fb);
          }
        }
      }
      // the last stages' copies have landed before the CTA may exit
      for (int pp = max(0, p - NST); pp < p; ++pp) mbar_drain(smem_u32(&bar_full[pp % NST]), uint32_t((pp / NST) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int p = 0, c = 0;
      bool ok = true;
      for (int it = 0; it < nitem_cta && ok; ++it) {
        for (int ch = 0; ch < nchunk && ok; ++ch, ++c) {
          if (c > 0 && !(ok = mbar_wait(smem_u32(&bar_acce), uint32_t((c - 1) & 1), abort))) break;
          fence_after();
          for (int h = 0; h < KBC; ++h, ++p) {
            const int s = p % NST;
            if (!(ok = mbar_wait(smem_u32(&bar_full[s]), uint32_t((p / NST) & 1), abort))) break;
            fence_after();
            const uint32_t sa = base + uint32_t(s) * STAGE, sb = sa + S * A_SLICE;
            mma_kstep(tmem, sa, sb, h == 0);
            mma_kstep(tmem, sa + 256, sb + 256, false);
            commit(smem_u32(&bar_empty[s]));
          }
          if (ok) commit(smem_u32(&bar_accf));
        }
      }
      // every MMA has completed before TMEM is freed
      commit(smem_u32(&bar_done));
      mbar_drain(smem_u32(&bar_done), 0);
    }
    __syncwarp();
  } else {
    // ---------------- flush warps ----------------
    const int quarter = warp & 3;                    // TMEM lanes 32 quarter .. + 31
    const int half = (warp - 2) >> 2;                // columns 32 half .. + 31
    const int rloc = 32 * quarter + lane;            // tile row of this thread
    const uint32_t trow = tmem + (uint32_t(32 * quarter) << 16);
    int c = 0;
    bool ok = true;
    for (int it = 0; it < nitem_cta && ok; ++it) {
      const int item = item0 + it * item_step;
      const int64_t m0 = int64_t(item / tiles_n) * BM, n0 = int64_t(item % tiles_n) * BN;
      dd master[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) master[j] = {0.f, 0.f};
      for (int ch = 0; ch < nchunk; ++ch, ++c) {
        const int64_t kc = (kb0 + ch * KBC) / KBC;
        const float fa = pow2(A.ex[kc * A.Mp + m0 + rloc] - 7);
        const float fbl = pow2(B.ex[kc * B.Mp + n0 + 32 * half + lane] - 7);
        if (!(ok = mbar_wait(smem_u32(&bar_accf), uint32_t(c & 1), abort))) break;
        fence_after();
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
          float v[6][16];
          tmem_ld_levels(trow + uint32_t(32 * half + 16 * sub), v);
          if (sub == 1) {  // TMEM read: the issuer may start the next chunk
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float hi, lo;
            combine_levels(v[0][j], v[1][j], v[2][j], v[3][j], v[4][j], v[5][j], hi, lo);
            const float fb = __shfl_sync(0xffffffffu, fbl, 16 * sub + j);
            add_scaled(master[16 * sub + j], hi, lo, fa * fb);
          }
        }
      }
      if (!ok) break;
      const int64_t r = m0 + rloc;
      const int64_t c0 = n0 + 32 * half;
      if (r < A.M) {
        // update: when the thread's 32 columns are one contiguous run of one
        // segment of Y, 16-byte aligned, write them as 16 two-element vectors
        bool fast = false;
        dd* yrow = nullptr;
        if (MODE == 1 && c0 + 32 <= B.M) {
          int sg = 0;
          while (sg + 1 < uo.Y.nseg && c0 >= uo.Y.start[sg + 1]) ++sg;
          yrow = uo.Y.ptr[sg] + r * uo.Y.ld[sg] + (c0 - uo.Y.start[sg]);
          fast = c0 + 32 <= uo.Y.start[sg + 1] && (reinterpret_cast<uintptr_t>(yrow) & 15) == 0;
        }
        if (fast) {
          float4* y4 = reinterpret_cast<float4*>(yrow);
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            dd v0 = master[j], v1 = master[j + 1];
            if (uo.has_beta) {
              const float4 old = y4[j / 2];
              dd_mac(v0, dd{old.x, old.y}, uo.beta);
              dd_mac(v1, dd{old.z, old.w}, uo.beta);
            }
            dd_renorm(v0);
            dd_renorm(v1);
            y4[j / 2] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t col = c0 + j;
            if (col < B.M) {
              if (MODE == 0) {
                go.part[int64_t(blockIdx.z) * A.M * B.M + r * B.M + col] =
                    double(master[j].hi) + double(master[j].lo);
              } else {
                dd* yp = uo.Y.at(r, int(col));
                dd v = master[j];
                if (uo.has_beta) dd_mac(v, *yp, uo.beta);
                dd_renorm(v);
                *yp = v;
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

template <int MODE>
cudaError_t set_smem5() {
  static thread_local int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev != dev) {
    e = cudaFuncSetAttribute(tc5_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM));
    if (e != cudaSuccess) return e;
    done_dev = dev;
  }
  return cudaSuccess;
}

int live_tiles(int a, int b, bool sym) {
  const int ta = (a + BM - 1) / BM, tb = (b + BN - 1) / BN;
  if (!sym) return ta * tb;
  int t = 0;
  for (int i = 0; i < ta; ++i)
    for (int j = 0; j < tb; ++j)
      if (!(j * BN + BN - 1 < i * BM)) ++t;
  return t;
}

}  // namespace

int tc5_gram_nsplit(int64_t n, int a, int b, bool sym) {
  int ns = num_sms() / std::max(1, live_tiles(a, b, sym));  // one CTA per SM, one wave
  const int64_t nch = cdiv(n, CH);
  if (ns > nch) ns = int(nch);
  if (ns < 1) ns = 1;
  return ns;
}

cudaError_t tc5_gram(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* scratch, int ns,
                     cudaStream_t st, const int* gate) {
  cudaError_t e = set_smem5<0>();
  if (e != cudaSuccess) return e;
  const int64_t nkb = nkb_of(n);
  const int64_t kb_per = cdiv(cdiv(n, CH), ns) * KBC;
  const int tm = (a + BM - 1) / BM, tn = (b + BN - 1) / BN;
  GramOut go{scratch, sym};
  UpdOut uo{};
  dim3 grid(tn, tm, ns);
  tc5_kernel<0><<<grid, THREADS, SMEM, st>>>(opnd(slu, n, a), opnd(slv, n, b), int(nkb), int(kb_per), tn, tm * tn,
                                             go, uo, gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tc5_update(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<dd>& Y, double beta,
                       cudaStream_t st, const int* gate) {
  cudaError_t e = set_smem5<1>();
  if (e != cudaSuccess) return e;
  const int64_t nkb = nkb_of(s);
  const int64_t tm = cdiv(n, BM);
  const int tn = (c + BN - 1) / BN;
  const int64_t items = tm * tn;
  int64_t grid = num_sms();
  if (grid > items) grid = items;
  GramOut go{};
  UpdOut uo;
  uo.Y = Y;
  const float bh = float(beta);
  uo.beta = dd{bh, float(beta - double(bh))};
  uo.has_beta = beta != 0.0;
  tc5_kernel<1><<<(unsigned)grid, THREADS, SMEM, st>>>(opnd(slu, s, n), opnd(slc, s, c), int(nkb), int(nkb), tn,
                                                       int(items), go, uo, gate);
  count_launches(1);
  return cudaGetLastError();
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
