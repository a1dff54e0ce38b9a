// Double-float block products on the tensor cores: the Gram products
// G = U^T V and the block updates Y = U C + beta Y of the Rayleigh-Ritz,
// orthogonalisation and update steps of arXiv:2409.05572 (Algorithms 1-3),
// the two contractions that dominate every iteration.
//
// Exact splitting, a fixed-point form of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012).  Both operands of a product P = A B^T
// (A: M x K, B: N x K, contraction over K) are cut into six integer slices
// against a power of two shared by one CHUNK of 128 consecutive K indices of
// one row of A (or B): with e the exponent of the chunk's largest |x|
// (max < 2^e),
//   x 2^(7 - e) = s_0 + s_1 2^-8 + ... + s_5 2^-40 + r,  |s_i| <= 128,
//   |r| <= 2^-41, i.e. r is below 2^-47 of the chunk's max.
// Integers of magnitude <= 256 are exact in bf16, every product s_i t_j
// (<= 2^14) is exact in the fp32 accumulators of mma.sync, and for every level
// l = i + j <= 5 the sum over one chunk (128 K indices) of its at most six
// products per index stays below 6 * 128 * 2^14 < 2^24, an integer that fp32
// represents exactly, so each level
// accumulates EXACTLY in its own fp32 accumulator, whatever order the tensor
// core adds in.  After every chunk the six level sums are combined into a
// double-float (two TwoSums, the small levels added into the low part: about
// 2^-44 of the largest possible chunk sum), scaled by 2^(e_a - 7) 2^(e_b - 7)
// (each factor a normal float for the exponents -99 .. 128 a chunk can have)
// and added to a double-float accumulator.  The levels l >= 6 are dropped
// (per K index at most 20 * 2^-48 of max|a| max|b| over the chunk) and six
// slices leave at most 2^-41 of the scaled value (another 8 * 2^-48): at most
// about 28 * 2^-48 per K index in all, about 2^-48 of it on average.  The
// result is accurate normwise (to the chunk maxima) rather than componentwise
// like the FP32-pipe double-float kernels.
//
//  Gram G = U^T V:   A = U^T, B = V^T, K = the n rows; chunks are 128 rows of
//                    one column (tc_slice_cols).
//  Update U C:       A = U, B = C^T, K = the s columns of U; chunks are 128
//                    columns of one row of U (tc_slice_rows) and 128 rows of one
//                    column of C (tc_slice_coef, from float64 C).
//
// The slice layout is described in tc.cuh.  Two product kernels read it:
// the tcgen05 kernel of k_tc5.cu (default) and, in this file, an mma.sync
// kernel (EIG_TC_KERNEL=mma selects it): it streams 32-K blocks of both
// operands into shared memory with cp.async (three stages), loads m16n8k16
// fragments with ldmatrix and issues 21 MMAs per fragment pair and k-step
// (all slice pairs with i + j <= 5).  Gram: split-K partial tiles, summed in
// a fixed order by the same reduction as the CUDA-core Gram.  Update:
// persistent CTAs walk the 64 x 64 output tiles, N fastest, and write
// Y = P + beta Y in double-float.
//
// Range: chunks whose maximum is below 2^-100 are treated as 0 (their
// products are below 2^-100 times the other operand, far under the rounding
// of any entry that matters); double-float itself has the float32 exponent
// range.
#include <cstdlib>
#include <cstring>

#include "blocks.cuh"
#include "tc.cuh"

namespace eig {

using namespace tc;

namespace {

constexpr int TC_T = 64;       // mma.sync CTA tile: 64 rows of A x 64 rows of B
constexpr int TC_KP = 40;      // padded pitch (bf16) of one row's 32 K values in shared memory
constexpr int TC_NST = 3;      // pipeline stages
constexpr int TC_OPND = S * TC_T * TC_KP;  // bf16 elements per operand and stage
constexpr int TC_STAGE = 2 * TC_OPND;
constexpr size_t TC_SHM = size_t(TC_NST) * TC_STAGE * sizeof(__nv_bfloat16);

// slices of one double-float value, scaled by `scale` (a power of two)
__device__ __forceinline__ void cut(float hv, float lv, float scale, float* s) {
  hv *= scale;
  lv *= scale;
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const float r = rintf(hv);
    s[q] = r;
    float nh, nl;
    two_sum(hv - r, lv, nh, nl);  // hv - r is exact (Sterbenz)
    hv = nh * 256.f;
    lv = nl * 256.f;
  }
}

__device__ __forceinline__ int chunk_exp(float mx) {
  int e = ZERO_EXP;
  if (mx >= 0x1p-100f) frexpf(mx, &e);  // 2^(e-1) <= mx < 2^e
  return e;
}

__device__ __forceinline__ float exp_scale(int e) { return e == ZERO_EXP ? 0.f : ldexpf(1.0f, 7 - e); }

// the 16 values v[0..15][q] of one row, K indices k0 .. k0 + 15 (k0 a
// multiple of 16) of one block -> two 16-byte core-matrix rows
__device__ __forceinline__ void store16(__nv_bfloat16* blk, int64_t r, int k0, const float (*v)[S], int q) {
  uint32_t p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i][q], v[2 * i + 1][q]);
    p[i] = *reinterpret_cast<const uint32_t*>(&b);
  }
  *reinterpret_cast<uint4*>(blk + in_block(r, k0)) = make_uint4(p[0], p[1], p[2], p[3]);
  *reinterpret_cast<uint4*>(blk + in_block(r, k0 + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
}

// ---------------------------------------------------------------------------
// Slicing.  CTA = one 64 x 64 square (one chunk x 64 operand rows), 256
// threads; staged through shared memory so that both the read of the
// row-major block and the write of the slice layout are coalesced.  The
// grids cover the padded operand rows, which get zero slices.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void col_lookup(const Blk<dd>& U, int c, const dd*& p, int64_t& ld) {
  int s = 0;
  while (s + 1 < U.nseg && c >= U.start[s + 1]) ++s;
  p = U.ptr[s] + (c - U.start[s]);
  ld = U.ld[s];
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

// Slicer squares: one 128-index chunk of K x 32 operand rows, 256 threads,
// two shared-memory buffers of 128 x 33 (COLS) or 32 x 129 (ROWS) float2.
constexpr int SQ_K = CH;   // 128
constexpr int SQ_M = 32;
constexpr int SL_P_COLS = SQ_M + 1, SL_P_ROWS = SQ_K + 1;
constexpr int SL_TILE = SQ_K * SQ_M + 128;  // float2 per buffer (either pitch fits)
constexpr size_t SL_SHM = size_t(2) * SL_TILE * sizeof(float2);

// Both slicers: persistent CTAs walk the squares (a, b) of U, item = a nb + b;
// the next square's 8-byte loads are in flight (cp.async, two shared-memory
// buffers) while the current one is cut.
//  COLS (Gram operand): K = rows of U, operand rows = columns of U; square =
//       rows 128 a .. + 127 x columns 32 b .. + 31; one exponent per
//       (128-row chunk a, column).
//  ROWS (update operand): K = columns of U, operand rows = rows of U; square
//       = rows 32 a .. + 31 x columns 128 b .. + 127; one exponent per
//       (row, 128-column chunk b).
template <bool COLS>
__global__ void __launch_bounds__(256) tc_slice_kernel(int64_t n, Blk<dd> U, Layout o, int64_t nb, int64_t items,
                                                       const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int P = COLS ? SL_P_COLS : SL_P_ROWS;
  constexpr int ROWS_SQ = COLS ? SQ_K : SQ_M;  // rows of U in a square
  constexpr int COLS_SQ = COLS ? SQ_M : SQ_K;  // columns of U in a square
  constexpr int LC = COLS_SQ, LR = 256 / COLS_SQ;  // loader: LC columns x LR rows per step
  extern __shared__ __align__(16) float2 sdraw[];
  __shared__ float pmax[8][32];
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
    const dd* colp = nullptr;
    int64_t cld = 0;
    if (c < w) col_lookup(U, c, colp, cld);
    float2* dst = sdraw + buf * SL_TILE;
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
    const float2* sd = sdraw + buf * SL_TILE;
    const int64_t a = item / nb, b = item % nb;
    if (COLS) {
      // column maxima over the 128 rows: 8 partial maxima per column
      const int lc = t & 31, lr = t >> 5;
      float m = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) m = fmaxf(m, fabsf(sd[(lr + 8 * i) * P + lc].x));
      pmax[lr][lc] = m;
      __syncthreads();
      if (t < 32) {
        float mm = pmax[0][t];
#pragma unroll
        for (int i = 1; i < 8; ++i) mm = fmaxf(mm, pmax[i][t]);
        const int e = chunk_exp(mm);
        sexp[t] = e;
        o.ex[a * o.Mp + b * SQ_M + t] = e == ZERO_EXP ? 0 : e;
      }
    } else {
      // row maxima over the 128 columns: 8 threads per row
      const int row = t >> 3, part = t & 7;
      float m = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) m = fmaxf(m, fabsf(sd[row * P + part + 8 * i].x));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
      if (part == 0) {
        const int e = chunk_exp(m);
        sexp[row] = e;
        o.ex[b * o.Mp + a * SQ_M + row] = e == ZERO_EXP ? 0 : e;
      }
    }
    __syncthreads();
    // thread -> (group g of 16 K indices, operand row idx of the square)
    const int g = t >> 5, idx = t & 31;
    const float scale = exp_scale(sexp[idx]);
    float v[16][S];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float2 x = COLS ? sd[(16 * g + i) * P + idx] : sd[idx * P + 16 * g + i];
      cut(x.x, x.y, scale, v[i]);
    }
    const int64_t kb = (COLS ? a : b) * KBC + (g >> 1);
    const int64_t orow = (COLS ? b : a) * SQ_M + idx;
#pragma unroll
    for (int q = 0; q < S; ++q) store16(o.sl + o.block(q, kb), orow, (g & 1) * 16, v, q);
    __syncthreads();  // the buffer is refilled by the next issue
    buf ^= 1;
  }
  cp_async_wait_s<0>();
}

// Update operand B from float64 C (s x c, ldc) times scale: K = rows of C,
// operand rows = columns of C.  Cut in float64 (exact: each step removes the
// integer part of a value with at most 53 significant bits).
__global__ void __launch_bounds__(256) tc_slice_coef_kernel(int s, int c, const double* __restrict__ C, int64_t ldc,
                                                            double scale, Layout o, const int* gate) {
  if (gate && *gate == 0) return;
  const int j0 = blockIdx.x * 32;
  const int kc = blockIdx.y;
  const int k00 = kc * CH;
  __shared__ double sc[CH][33];
  __shared__ double pmax[8][32];
  __shared__ int sexp[32];
  const int t = threadIdx.x;
  {
    const int lj = t & 31, lk = t >> 5;
    const int j = j0 + lj;
    double m = 0.0;
    for (int i = 0; i < CH / 8; ++i) {
      const int kk = lk + 8 * i;
      const int k = k00 + kk;
      const double x = (j < c && k < s) ? scale * C[int64_t(k) * ldc + j] : 0.0;
      sc[kk][lj] = x;
      m = fmax(m, fabs(x));
    }
    pmax[lk][lj] = m;
  }
  __syncthreads();
  if (t < 32) {
    double mm = pmax[0][t];
    for (int i = 1; i < 8; ++i) mm = fmax(mm, pmax[i][t]);
    int e = ZERO_EXP;
    if (mm >= 0x1p-100) frexp(mm, &e);
    sexp[t] = e;
    o.ex[int64_t(kc) * o.Mp + j0 + t] = e == ZERO_EXP ? 0 : e;
  }
  __syncthreads();
  const int g = t >> 5, col = t & 31;
  const int e = sexp[col];
  float v[16][S];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    double x = e == ZERO_EXP ? 0.0 : ldexp(sc[16 * g + i][col], 7 - e);
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const double r = rint(x);
      v[i][q] = float(r);
      x = (x - r) * 256.0;
    }
  }
  const int64_t kb = int64_t(kc) * KBC + (g >> 1);
#pragma unroll
  for (int q = 0; q < S; ++q) store16(o.sl + o.block(q, kb), j0 + col, (g & 1) * 16, v, q);
}

// ---------------------------------------------------------------------------
// mma.sync product kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// MODE 0: Gram (one item per CTA: tile (blockIdx.y, blockIdx.x), K blocks
// [z * kb_per, (z + 1) * kb_per) of split z = blockIdx.z).
// MODE 1: update (persistent: items t = blockIdx.x + i * gridDim.x over the
// tiles_m x tiles_n output tiles, N fastest, all K blocks).
template <int MODE>
__global__ void __launch_bounds__(512, 1) tc_product_kernel(Opnd A, Opnd B, int nkb, int kb_per, int tiles_n,
                                                            int nitems, GramOut go, UpdOut uo, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int am = (warp >> 2) * 16;  // warp's 16 A rows within the tile
  const int bn = (warp & 3) * 16;   // warp's 16 B rows within the tile
  const int g = lane >> 2, tq = lane & 3;

  // this CTA's sequence of (item, K block) positions
  int item0, item_step, nitem_cta, kb0, nkb_item;
  if (MODE == 0) {
    if (go.sym && blockIdx.y > blockIdx.x) return;
    item0 = int(blockIdx.y) * tiles_n + int(blockIdx.x);
    item_step = 1;
    nitem_cta = 1;
    kb0 = int(blockIdx.z) * kb_per;
    const int kb1 = min(kb0 + kb_per, nkb);
    nkb_item = kb1 > kb0 ? kb1 - kb0 : 0;
  } else {
    item0 = blockIdx.x;
    item_step = gridDim.x;
    nitem_cta = item0 < nitems ? (nitems - 1 - item0) / item_step + 1 : 0;
    kb0 = 0;
    nkb_item = nkb;
  }
  if (nkb_item == 0 && MODE == 1) nitem_cta = 0;

  // operand rows are padded to a multiple of 128 with zero slices, so every
  // 64-row tile is in bounds
  auto load_stage = [&](int it, int kbi, int buf) {
    const int item = item0 + it * item_step;
    const int64_t kb = kb0 + kbi;
    const int64_t m0 = int64_t(item / tiles_n) * TC_T, n0 = int64_t(item % tiles_n) * TC_T;
    __nv_bfloat16* dst = sm + buf * TC_STAGE;
#pragma unroll
    for (int i = 0; i < (S * TC_T * 4) / 512; ++i) {
      const int id = t + 512 * i;
      const int q = id / (TC_T * 4);
      const int rem = id % (TC_T * 4);
      const int col = rem >> 2, piece = rem & 3;
      const __nv_bfloat16* ga = A.sl + (int64_t(q) * nkb + kb) * A.Mp * KB + in_block(m0 + col, piece * 8);
      const __nv_bfloat16* gb = B.sl + (int64_t(q) * nkb + kb) * B.Mp * KB + in_block(n0 + col, piece * 8);
      cp_async16(dst + (q * TC_T + col) * TC_KP + piece * 8, ga);
      cp_async16(dst + TC_OPND + (q * TC_T + col) * TC_KP + piece * 8, gb);
    }
  };

  // ldmatrix row addresses (element offsets within a stage)
  const int lm = lane >> 3, lr = lane & 7;
  const int a_off = (am + lr + (lm & 1) * 8) * TC_KP + (lm >> 1) * 8;
  const int b_off = TC_OPND + (bn + (lm >> 1) * 8 + lr) * TC_KP + (lm & 1) * 8;

  float acc[2][6][4];
  dd master[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int f = 0; f < 4; ++f) master[j][f] = {0.f, 0.f};

  // load position (ld_it, ld_k) runs TC_NST - 1 stages ahead of compute
  int ld_it = 0, ld_k = 0, ld_buf = 0;
#pragma unroll
  for (int s = 0; s < TC_NST - 1; ++s) {
    if (ld_it < nitem_cta && nkb_item > 0) {
      load_stage(ld_it, ld_k, ld_buf);
      if (++ld_k == nkb_item) {
        ld_k = 0;
        ++ld_it;
      }
      ld_buf = ld_buf + 1 == TC_NST ? 0 : ld_buf + 1;
    }
    cp_async_commit();
  }
  int buf = 0;
  for (int it = 0; it < nitem_cta; ++it) {
    const int item = item0 + it * item_step;
    const int64_t m0 = int64_t(item / tiles_n) * TC_T, n0 = int64_t(item % tiles_n) * TC_T;
    const int64_t rl = m0 + am + g, rh = rl + 8;
    for (int kbi = 0; kbi < nkb_item; ++kbi) {
      const int kb = kb0 + kbi;
      if (kb % KBC == 0 || kbi == 0) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int l = 0; l < 6; ++l)
#pragma unroll
            for (int f = 0; f < 4; ++f) acc[j][l][f] = 0.f;
      }
      cp_async_wait<TC_NST - 2>();
      __syncthreads();
      if (ld_it < nitem_cta) {
        load_stage(ld_it, ld_k, ld_buf);
        if (++ld_k == nkb_item) {
          ld_k = 0;
          ++ld_it;
        }
        ld_buf = ld_buf + 1 == TC_NST ? 0 : ld_buf + 1;
      }
      cp_async_commit();
      const __nv_bfloat16* stg = sm + buf * TC_STAGE;
      buf = buf + 1 == TC_NST ? 0 : buf + 1;
#pragma unroll
      for (int ks = 0; ks < KB; ks += 16) {
        uint32_t bf[S][4];
#pragma unroll
        for (int q = 0; q < S; ++q) ldsm_x4(bf[q], stg + b_off + q * TC_T * TC_KP + ks);
#pragma unroll
        for (int qi = 0; qi < S; ++qi) {
          uint32_t af[4];
          ldsm_x4(af, stg + a_off + qi * TC_T * TC_KP + ks);
#pragma unroll
          for (int qj = 0; qj < S - qi; ++qj) {
            mma_bf16(acc[0][qi + qj], af, bf[qj][0], bf[qj][1]);
            mma_bf16(acc[1][qi + qj], af, bf[qj][2], bf[qj][3]);
          }
        }
      }
      const bool last = kbi + 1 == nkb_item;
      if (kb % KBC == KBC - 1 || last) {
        // chunk done: value = sum_l acc_l 2^(-8 l) (exact integers per
        // level), times 2^(e_a - 7) 2^(e_b - 7), into the double-float master
        const int64_t kc = kb / KBC;
        const float fal = pow2(A.ex[kc * A.Mp + rl] - 7);
        const float fah = pow2(A.ex[kc * A.Mp + rh] - 7);
        float fbc[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) fbc[f] = pow2(B.ex[kc * B.Mp + n0 + bn + 8 * (f >> 1) + 2 * tq + (f & 1)] - 7);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            float hi, lo;
            combine_levels(acc[j][0][f], acc[j][1][f], acc[j][2][f], acc[j][3][f], acc[j][4][f], acc[j][5][f], hi,
                           lo);
            add_scaled(master[j][f], hi, lo, (f >= 2 ? fah : fal) * fbc[2 * j + (f & 1)]);
          }
      }
    }
    // item done: write it out
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int64_t r = f >= 2 ? rh : rl;
        const int64_t c = n0 + bn + 8 * j + 2 * tq + (f & 1);
        if (r < A.M && c < B.M) {
          if (MODE == 0) {
            go.part[int64_t(blockIdx.z) * A.M * B.M + r * B.M + c] =
                double(master[j][f].hi) + double(master[j][f].lo);
          } else {
            dd* yp = uo.Y.at(r, int(c));
            dd v = master[j][f];
            if (uo.has_beta) dd_mac(v, *yp, uo.beta);
            dd_renorm(v);
            *yp = v;
          }
        }
        master[j][f] = {0.f, 0.f};
      }
  }
  cp_async_wait<0>();
}

int gram_tc_nsplit(int64_t n, int a, int b, bool sym) {
  const int ta = (a + TC_T - 1) / TC_T, tb = (b + TC_T - 1) / TC_T;
  const int tiles = (sym && ta == tb) ? ta * (ta + 1) / 2 : ta * tb;
  int ns = num_sms() / tiles;  // one CTA per SM, one wave
  const int64_t nch = cdiv(n, CH);
  if (ns > nch) ns = int(nch);
  if (ns < 1) ns = 1;
  return ns;
}

template <int MODE>
cudaError_t set_smem() {
  static thread_local int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev != dev) {
    e = cudaFuncSetAttribute(tc_product_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC_SHM));
    if (e != cudaSuccess) return e;
    done_dev = dev;
  }
  return cudaSuccess;
}

// EIG_TC_KERNEL=mma selects the mma.sync product kernel
bool use_mma_sync() {
  static const bool v = [] {
    const char* e = std::getenv("EIG_TC_KERNEL");
    return e && std::strcmp(e, "mma") == 0;
  }();
  return v;
}

UpdOut upd_out(const Blk<dd>& Y, double beta) {
  UpdOut uo;
  uo.Y = Y;
  const float bh = float(beta);
  uo.beta = dd{bh, float(beta - double(bh))};
  uo.has_beta = beta != 0.0;
  return uo;
}

}  // namespace

// the slicers use 33-35 KB of shared memory per 256-thread CTA: ask for the
// largest shared-memory carveout so that six CTAs fit on an SM
template <typename K>
void max_carveout(K kernel) {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || done_dev == dev) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  done_dev = dev;
}

size_t tc_slice_bytes(int64_t K, int64_t M) {
  const size_t mp = size_t(mpad_of(M));
  const size_t sb = sizeof(__nv_bfloat16) * size_t(S) * size_t(nkb_of(K)) * mp * KB;
  return sb + sizeof(int) * size_t(cdiv(K, CH)) * mp;
}

size_t gram_tc_scratch_elems(int64_t n, int a, int b, bool sym) {
  const int ns = std::max(gram_tc_nsplit(n, a, b, sym), tc5_gram_nsplit(n, a, b, sym));
  return size_t(ns) * size_t(a) * size_t(b);
}

template <bool COLS>
cudaError_t slice_launch(int64_t n, const Blk<dd>& U, const Layout& o, int64_t na, int64_t nb, cudaStream_t st,
                         const int* gate) {
  static thread_local int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev != dev) {
    e = cudaFuncSetAttribute(tc_slice_kernel<COLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SL_SHM));
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(tc_slice_kernel<COLS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    done_dev = dev;
  }
  const int64_t items = na * nb;
  int64_t grid = int64_t(num_sms()) * 3;  // three 67 KB CTAs per SM
  if (grid > items) grid = items;
  tc_slice_kernel<COLS><<<(unsigned)grid, 256, SL_SHM, st>>>(n, U, o, nb, items, gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tc_slice_cols(int64_t n, const Blk<dd>& U, void* buf, cudaStream_t st, const int* gate) {
  const int w = U.width;
  if (w <= 0 || n <= 0) return cudaSuccess;
  const Layout o = layout(buf, n, w);
  // squares: 128-row chunks of U (K) x 32-column blocks (operand rows, padded)
  return slice_launch<true>(n, U, o, cdiv(n, CH), o.Mp / SQ_M, st, gate);
}

cudaError_t tc_slice_rows(int64_t n, const Blk<dd>& U, void* buf, cudaStream_t st, const int* gate) {
  const int w = U.width;
  if (w <= 0 || n <= 0) return cudaSuccess;
  const Layout o = layout(buf, w, n);
  // squares: 32-row blocks of U (operand rows, padded) x 128-column chunks (K)
  return slice_launch<false>(n, U, o, o.Mp / SQ_M, cdiv(w, CH), st, gate);
}

cudaError_t tc_slice_coef(int s, int c, const double* C, int64_t ldc, double scale, void* buf, cudaStream_t st,
                          const int* gate) {
  if (s <= 0 || c <= 0) return cudaSuccess;
  const Layout o = layout(buf, s, c);
  dim3 grid((unsigned)(o.Mp / 32), (unsigned)cdiv(s, CH));
  max_carveout(tc_slice_coef_kernel);
  tc_slice_coef_kernel<<<grid, 256, 0, st>>>(s, c, C, ldc, scale, o, gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gram_tc_product(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* G,
                            int64_t ldg, double* scratch, cudaStream_t st, const int* gate) {
  if (a <= 0 || b <= 0 || n <= 0) return cudaSuccess;
  int ns;
  if (use_mma_sync()) {
    cudaError_t e = set_smem<0>();
    if (e != cudaSuccess) return e;
    const int64_t nkb = nkb_of(n);
    ns = gram_tc_nsplit(n, a, b, sym);
    const int64_t kb_per = cdiv(cdiv(n, CH), ns) * KBC;
    const int tm = (a + TC_T - 1) / TC_T, tn = (b + TC_T - 1) / TC_T;
    GramOut go{scratch, sym};
    UpdOut uo{};
    dim3 grid(tn, tm, ns);
    tc_product_kernel<0><<<grid, 512, TC_SHM, st>>>(opnd(slu, n, a), opnd(slv, n, b), int(nkb), int(kb_per), tn,
                                                    tm * tn, go, uo, gate);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    ns = tc5_gram_nsplit(n, a, b, sym);
    cudaError_t e = tc5_gram(n, a, b, slu, slv, sym, scratch, ns, st, gate);
    if (e != cudaSuccess) return e;
  }
  return gram_reduce(a, b, ns, sym, scratch, G, ldg, st, gate);
}

cudaError_t update_tc_product(int64_t n, int s, int c, const void* slu, const void* slc, const Blk<dd>& Y,
                              double beta, cudaStream_t st, const int* gate) {
  if (n <= 0 || c <= 0) return cudaSuccess;
  if (!use_mma_sync()) return tc5_update(n, s, c, slu, slc, Y, beta, st, gate);
  cudaError_t e = set_smem<1>();
  if (e != cudaSuccess) return e;
  const int64_t nkb = nkb_of(s);
  const int64_t tm = cdiv(n, TC_T);
  const int tn = (c + TC_T - 1) / TC_T;
  const int64_t items = tm * tn;
  int64_t grid = num_sms();
  if (grid > items) grid = items;
  GramOut go{};
  tc_product_kernel<1><<<(unsigned)grid, 512, TC_SHM, st>>>(opnd(slu, s, n), opnd(slc, s, c), int(nkb), int(nkb),
                                                            tn, int(items), go, upd_out(Y, beta), gate);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace eig
