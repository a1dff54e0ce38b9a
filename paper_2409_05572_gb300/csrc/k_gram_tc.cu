// Tensor-core Gram product G = U^T V for double-float blocks: the dominant
// contraction of the Rayleigh-Ritz and orthogonalisation steps of
// arXiv:2409.05572 (Algorithms 1-3).
//
// Exact splitting, a fixed-point form of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012).  For every chunk of 128 rows and every column
// the double-float values x = hi + lo are scaled by 2^(7 - e), e the exponent
// of the chunk's largest |hi| (max < 2^e), and cut into six integer slices
//   x 2^(7 - e) = s_0 + s_1 2^-8 + ... + s_5 2^-40 + r,  |s_i| <= 128,
//   |r| <= 2^-41, i.e. r is below 2^-47 of the chunk's max.
// Integers of magnitude <= 256 are exact in bf16, every product s_i t_j
// (<= 2^14) is exact in the fp32 accumulators of mma.sync, and for every level
// l = i + j <= 5 the sum over 64 rows of its at most six products per row
// stays below 6 * 64 * 2^14 < 2^23, so each level accumulates EXACTLY in its
// own fp32 accumulator, whatever order the tensor core adds in.  Every 64
// rows the six level sums are combined into a double-float (TwoSum), scaled by
// 2^(e_u + e_v - 14) and added to a double-float accumulator.  The levels
// l >= 6 are dropped: per row that is at most 20 * 2^-48 of
// max|u| max|v| over the chunk, and about 2^-48 of it on average.
//
// Pass 1 (tc_slice_kernel) writes the slices in the order the product reads
// them, [slice][32-row block][column][32 rows] bf16, and one exponent per
// (128-row chunk, column).  Pass 2 (gram_tc_kernel) streams 32-row blocks of
// both operands into shared memory with cp.async (three stages), loads
// m16n8k16 fragments with ldmatrix and issues 21 MMAs per fragment pair and
// k-step (all slice pairs with i + j <= 5).  Split-K partial tiles are summed
// in a fixed order by the same reduction as the CUDA-core Gram.
//
// Range: entries whose chunk-column maximum is below 2^-100 are treated as 0
// (their products are below 2^-100 times the other operand, far under the
// double-float rounding of any entry that matters); the double-float format
// itself has the float32 exponent range.
#include <cuda_bf16.h>

#include "blocks.cuh"

namespace eig {

namespace {

constexpr int TC_S = 6;        // slices per value
constexpr int TC_RB = 32;      // rows per block (one pipeline stage)
constexpr int TC_CHUNK = 128;  // rows sharing one exponent per column
constexpr int TC_RBC = TC_CHUNK / TC_RB;
constexpr int TC_FLUSH = 2;    // row blocks (64 rows) between exact-level flushes
constexpr int TC_T = 64;       // CTA tile: 64 columns of U x 64 columns of V
constexpr int TC_KP = 40;      // padded pitch (bf16) of one column's 32 rows in shared memory
constexpr int TC_NST = 3;      // pipeline stages
constexpr int TC_OPND = TC_S * TC_T * TC_KP;  // bf16 elements per operand and stage
constexpr int TC_STAGE = 2 * TC_OPND;
constexpr size_t TC_SHM = size_t(TC_NST) * TC_STAGE * sizeof(__nv_bfloat16);
constexpr int TC_ZERO = -1000;  // exponent mark of an all-zero chunk column

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// ---------------------------------------------------------------------------
// pass 1: exponents and slices.  CTA = one 128-row chunk x 32 columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tc_slice_kernel(int64_t n, Blk<dd> U, int64_t nrb,
                                                       __nv_bfloat16* __restrict__ sl, int* __restrict__ ex,
                                                       const int* gate) {
  if (gate && *gate == 0) return;
  const int w = U.width;
  const int c0 = blockIdx.x * 32;
  const int chunk = blockIdx.y;
  const int64_t r0 = int64_t(chunk) * TC_CHUNK;
  __shared__ float shi[TC_CHUNK][33];
  __shared__ float slo[TC_CHUNK][33];
  __shared__ float pmax[8][32];
  __shared__ int sexp[32];
  const int t = threadIdx.x;
  {
    const int lc = t & 31, lr = t >> 5;
    const int c = c0 + lc;
    const dd* colp = nullptr;
    int64_t cld = 0;
    if (c < w) {
      int s = 0;
      while (s + 1 < U.nseg && c >= U.start[s + 1]) ++s;
      colp = U.ptr[s] + (c - U.start[s]);
      cld = U.ld[s];
    }
    float m = 0.f;
#pragma unroll 4
    for (int i = 0; i < TC_CHUNK / 8; ++i) {
      const int rr = lr + 8 * i;
      const int64_t r = r0 + rr;
      dd x = {0.f, 0.f};
      if (colp && r < n) x = colp[r * cld];
      shi[rr][lc] = x.hi;
      slo[rr][lc] = x.lo;
      m = fmaxf(m, fabsf(x.hi));
    }
    pmax[lr][lc] = m;
  }
  __syncthreads();
  if (t < 32) {
    float mm = pmax[0][t];
#pragma unroll
    for (int i = 1; i < 8; ++i) mm = fmaxf(mm, pmax[i][t]);
    int e = TC_ZERO;
    if (mm >= 0x1p-100f) frexpf(mm, &e);  // 2^(e-1) <= mm < 2^e
    sexp[t] = e;
    if (c0 + t < w) ex[int64_t(chunk) * w + c0 + t] = e == TC_ZERO ? 0 : e;
  }
  __syncthreads();
  // thread -> (row block rbl, column col, rows k0 .. k0 + 15)
  const int rbl = t >> 6, col = (t & 63) >> 1, k0 = (t & 1) * 16;
  const int c = c0 + col;
  if (c >= w) return;
  const int e = sexp[col];
  const float scale = e == TC_ZERO ? 0.f : ldexpf(1.0f, 7 - e);
  uint32_t packed[TC_S][8];
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    float s2[2][TC_S];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      float hv = shi[rbl * TC_RB + k0 + i + u][col] * scale;
      float lv = slo[rbl * TC_RB + k0 + i + u][col] * scale;
#pragma unroll
      for (int q = 0; q < TC_S; ++q) {
        const float s = rintf(hv);
        s2[u][q] = s;
        float nh, nl;
        two_sum(hv - s, lv, nh, nl);  // hv - s is exact (Sterbenz)
        hv = nh * 256.f;
        lv = nl * 256.f;
      }
    }
#pragma unroll
    for (int q = 0; q < TC_S; ++q) {
      const __nv_bfloat162 p = __floats2bfloat162_rn(s2[0][q], s2[1][q]);
      packed[q][i / 2] = *reinterpret_cast<const uint32_t*>(&p);
    }
  }
  const int64_t rb = int64_t(chunk) * TC_RBC + rbl;
#pragma unroll
  for (int q = 0; q < TC_S; ++q) {
    uint4* dst = reinterpret_cast<uint4*>(sl + ((int64_t(q) * nrb + rb) * w + c) * TC_RB + k0);
    dst[0] = make_uint4(packed[q][0], packed[q][1], packed[q][2], packed[q][3]);
    dst[1] = make_uint4(packed[q][4], packed[q][5], packed[q][6], packed[q][7]);
  }
}

// ---------------------------------------------------------------------------
// pass 2: tensor-core Gram on the slices
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int nb = pred ? 16 : 0;  // 0: zero-fill, nothing read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(nb));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__global__ void __launch_bounds__(512, 1) gram_tc_kernel(int a, int b, int64_t nrb, int64_t rb_per_split,
                                                         const __nv_bfloat16* __restrict__ su,
                                                         const int* __restrict__ eu,
                                                         const __nv_bfloat16* __restrict__ sv,
                                                         const int* __restrict__ ev, bool sym,
                                                         double* __restrict__ part, const int* gate) {
  if (gate && *gate == 0) return;
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (sym && tm > tn) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
  const int m0 = tm * TC_T, n0 = tn * TC_T;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int am = (warp >> 2) * 16;  // warp's 16 U columns within the tile
  const int bn = (warp & 3) * 16;   // warp's 16 V columns within the tile
  const int g = lane >> 2, tq = lane & 3;
  const int64_t rb_begin = int64_t(blockIdx.z) * rb_per_split;
  int64_t rb_end = rb_begin + rb_per_split;
  if (rb_end > nrb) rb_end = nrb;
  const int nblk = rb_end > rb_begin ? int(rb_end - rb_begin) : 0;

  // loader: per stage and operand TC_S x 64 columns x 4 pieces of 16 bytes
  auto load_stage = [&](int64_t rb, int buf) {
    __nv_bfloat16* dst = sm + buf * TC_STAGE;
#pragma unroll
    for (int i = 0; i < (TC_S * TC_T * 4) / 512; ++i) {
      const int id = t + 512 * i;
      const int q = id / (TC_T * 4);
      const int rem = id % (TC_T * 4);
      const int col = rem >> 2, piece = rem & 3;
      const int cu = m0 + col, cv = n0 + col;
      const __nv_bfloat16* gu = su + ((int64_t(q) * nrb + rb) * a + (cu < a ? cu : 0)) * TC_RB + piece * 8;
      const __nv_bfloat16* gv = sv + ((int64_t(q) * nrb + rb) * b + (cv < b ? cv : 0)) * TC_RB + piece * 8;
      cp_async16(dst + (q * TC_T + col) * TC_KP + piece * 8, gu, cu < a);
      cp_async16(dst + TC_OPND + (q * TC_T + col) * TC_KP + piece * 8, gv, cv < b);
    }
  };

  // ldmatrix row addresses (element offsets within a stage)
  const int lm = lane >> 3, lr = lane & 7;
  const int a_off = (am + lr + (lm & 1) * 8) * TC_KP + (lm >> 1) * 8;
  const int b_off = TC_OPND + (bn + (lm >> 1) * 8 + lr) * TC_KP + (lm & 1) * 8;

  // output coordinates of this thread's fragments
  const int r_lo = m0 + am + g, r_hi = r_lo + 8;
  int cidx[4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int u = 0; u < 2; ++u) cidx[2 * j + u] = n0 + bn + 8 * j + 2 * tq + u;

  float acc[2][6][4];
  dd master[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int f = 0; f < 4; ++f) master[j][f] = {0.f, 0.f};

#pragma unroll
  for (int s = 0; s < TC_NST - 1; ++s) {
    if (s < nblk) load_stage(rb_begin + s, s);
    cp_async_commit();
  }
  for (int it = 0; it < nblk; ++it) {
    const int64_t rb = rb_begin + it;
    if (it % TC_FLUSH == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int l = 0; l < 6; ++l)
#pragma unroll
          for (int f = 0; f < 4; ++f) acc[j][l][f] = 0.f;
    }
    cp_async_wait<TC_NST - 2>();
    __syncthreads();
    if (it + TC_NST - 1 < nblk) load_stage(rb + TC_NST - 1, (it + TC_NST - 1) % TC_NST);
    cp_async_commit();
    const __nv_bfloat16* stg = sm + (it % TC_NST) * TC_STAGE;
#pragma unroll
    for (int ks = 0; ks < TC_RB; ks += 16) {
      uint32_t bf[TC_S][4];
#pragma unroll
      for (int q = 0; q < TC_S; ++q) ldsm_x4(bf[q], stg + b_off + q * TC_T * TC_KP + ks);
#pragma unroll
      for (int qi = 0; qi < TC_S; ++qi) {
        uint32_t af[4];
        ldsm_x4(af, stg + a_off + qi * TC_T * TC_KP + ks);
#pragma unroll
        for (int qj = 0; qj < TC_S - qi; ++qj) {
          mma_bf16(acc[0][qi + qj], af, bf[qj][0], bf[qj][1]);
          mma_bf16(acc[1][qi + qj], af, bf[qj][2], bf[qj][3]);
        }
      }
    }
    if (it % TC_FLUSH == TC_FLUSH - 1 || it + 1 == nblk) {
      // value = sum_l acc_l 2^(-8 l) (exact integers per level), times
      // 2^(e_u + e_v - 14), added to the double-float master
      const int64_t chunk = rb / TC_RBC;
      const int eul = r_lo < a ? eu[chunk * a + r_lo] : 0;
      const int euh = r_hi < a ? eu[chunk * a + r_hi] : 0;
      int evc[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) evc[f] = cidx[f] < b ? ev[chunk * b + cidx[f]] : 0;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          float hi = acc[j][5][f], lo = 0.f;
#pragma unroll
          for (int l = 4; l >= 0; --l) {
            hi *= 0x1p-8f;
            lo *= 0x1p-8f;
            float s, e;
            two_sum(acc[j][l][f], hi, s, e);
            lo += e;
            hi = s;
          }
          const int sc = (f >= 2 ? euh : eul) + evc[2 * j + (f & 1)] - 14;
          hi = ldexpf(hi, sc);
          lo = ldexpf(lo, sc);
          float s, e;
          two_sum(master[j][f].hi, hi, s, e);
          e += master[j][f].lo + lo;
          master[j][f].hi = s + e;
          master[j][f].lo = e - (master[j][f].hi - s);
        }
    }
  }
  cp_async_wait<0>();
  double* out = part + int64_t(blockIdx.z) * a * b;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int r = f >= 2 ? r_hi : r_lo;
      const int c = cidx[2 * j + (f & 1)];
      if (r < a && c < b) out[int64_t(r) * b + c] = double(master[j][f].hi) + double(master[j][f].lo);
    }
}

int64_t tc_nrb(int64_t n) { return cdiv(n, TC_CHUNK) * TC_RBC; }

int gram_tc_nsplit(int64_t n, int a, int b, bool sym) {
  const int ta = (a + TC_T - 1) / TC_T, tb = (b + TC_T - 1) / TC_T;
  const int tiles = (sym && ta == tb) ? ta * (ta + 1) / 2 : ta * tb;
  int ns = num_sms() / tiles;  // one CTA per SM, one wave
  const int64_t nch = cdiv(n, TC_CHUNK);
  if (ns > nch) ns = int(nch);
  if (ns < 1) ns = 1;
  return ns;
}

}  // namespace

size_t gram_tc_slice_bytes(int64_t n, int w) {
  const size_t sb = sizeof(__nv_bfloat16) * size_t(TC_S) * size_t(tc_nrb(n)) * size_t(w) * TC_RB;
  return sb + sizeof(int) * size_t(cdiv(n, TC_CHUNK)) * size_t(w);
}

size_t gram_tc_scratch_elems(int64_t n, int a, int b, bool sym) {
  return size_t(gram_tc_nsplit(n, a, b, sym)) * size_t(a) * size_t(b);
}

cudaError_t gram_tc_slice(int64_t n, const Blk<dd>& U, void* slices, cudaStream_t st, const int* gate) {
  const int w = U.width;
  if (w <= 0 || n <= 0) return cudaSuccess;
  const int64_t nrb = tc_nrb(n);
  auto* sl = static_cast<__nv_bfloat16*>(slices);
  int* ex = reinterpret_cast<int*>(sl + size_t(TC_S) * size_t(nrb) * size_t(w) * TC_RB);
  dim3 grid((w + 31) / 32, (unsigned)cdiv(n, TC_CHUNK));
  tc_slice_kernel<<<grid, 256, 0, st>>>(n, U, nrb, sl, ex, gate);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gram_tc_product(int64_t n, int a, int b, const void* slu, const void* slv, bool sym, double* G,
                            int64_t ldg, double* scratch, cudaStream_t st, const int* gate) {
  if (a <= 0 || b <= 0 || n <= 0) return cudaSuccess;
  const int64_t nrb = tc_nrb(n);
  const auto* su = static_cast<const __nv_bfloat16*>(slu);
  const auto* sv = static_cast<const __nv_bfloat16*>(slv);
  const int* eu = reinterpret_cast<const int*>(su + size_t(TC_S) * size_t(nrb) * size_t(a) * TC_RB);
  const int* ev = reinterpret_cast<const int*>(sv + size_t(TC_S) * size_t(nrb) * size_t(b) * TC_RB);
  const int ns = gram_tc_nsplit(n, a, b, sym);
  const int64_t rbps = cdiv(cdiv(n, TC_CHUNK), ns) * TC_RBC;
  static thread_local int attr_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC_SHM));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  dim3 grid((b + TC_T - 1) / TC_T, (a + TC_T - 1) / TC_T, ns);
  gram_tc_kernel<<<grid, 512, TC_SHM, st>>>(a, b, nrb, rbps, su, eu, sv, ev, sym, scratch, gate);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return gram_reduce(a, b, ns, sym, scratch, G, ldg, st, gate);
}

}  // namespace eig
