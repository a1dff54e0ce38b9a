// n-sized block kernels of the eigensolvers (arXiv:2409.05572, Algorithms 1
// and 3): CSR SpMM (A X, A W, A S_drop, Chebyshev steps), split-K Gram
// products (X^T A X, S^T A S, [X,P]^T W, W^T W), block updates (X <- S C,
// W <- W - Q C, W <- W R^{-1}) and the residual / norm pass of Eq. conv.
//
// All are HBM- or FP32-pipe-bound streaming kernels over row-major blocks.
// In the double-float (DF64) form no FP64 instruction executes inside an
// n-sized loop: blocks are stored as {hi, lo} float pairs and every product
// is an FP32 TwoProd plus cross terms.
#include <atomic>
#include <cstdio>

#include "blocks.cuh"

namespace eig {

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s = p + e;
  return {s, e - (s - p)};
}

template <typename T> __device__ __forceinline__ T shfl_t(unsigned mask, T v, int src, int width);
template <> __device__ __forceinline__ double shfl_t<double>(unsigned m, double v, int s, int w) {
  return __shfl_sync(m, v, s, w);
}
template <> __device__ __forceinline__ float shfl_t<float>(unsigned m, float v, int s, int w) {
  return __shfl_sync(m, v, s, w);
}
template <> __device__ __forceinline__ dd shfl_t<dd>(unsigned m, dd v, int s, int w) {
  return {__shfl_sync(m, v.hi, s, w), __shfl_sync(m, v.lo, s, w)};
}

// accumulator initialised from a stored element
template <Arith A> __device__ __forceinline__ typename Pol<A>::Acc acc_from(typename Pol<A>::T x);
template <> __device__ __forceinline__ double acc_from<Arith::F64>(double x) { return x; }
template <> __device__ __forceinline__ dd acc_from<Arith::DF64>(dd x) { return x; }
template <> __device__ __forceinline__ float acc_from<Arith::F32>(float x) { return x; }
template <> __device__ __forceinline__ dd acc_from<Arith::C32>(float x) { return {x, 0.f}; }

// staged coefficient from a host double (host-side split for DF64)
template <Arith A> typename Pol<A>::S host_coef(double x);
template <> double host_coef<Arith::F64>(double x) { return x; }
template <> dd host_coef<Arith::DF64>(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
template <> float host_coef<Arith::F32>(double x) { return (float)x; }
template <> float host_coef<Arith::C32>(double x) { return (float)x; }

// product of a stored matrix value and a staged coefficient, as staged
template <Arith A> __device__ __forceinline__ typename Pol<A>::S scale_val(typename Pol<A>::T v,
                                                                          typename Pol<A>::S a);
template <> __device__ __forceinline__ double scale_val<Arith::F64>(double v, double a) { return v * a; }
template <> __device__ __forceinline__ dd scale_val<Arith::DF64>(dd v, dd a) { return dd_mul(v, a); }
template <> __device__ __forceinline__ float scale_val<Arith::F32>(float v, float a) { return v * a; }
template <> __device__ __forceinline__ float scale_val<Arith::C32>(float v, float a) { return v * a; }

// ---------------------------------------------------------------------------
// K1 / K10: CSR SpMM with a three-term epilogue.
// G lanes own one row; lane g covers column vectors g, g+G, ... (VEC elements
// each, 16-byte loads when VEC > 1).  The row's (colind, value) pairs are
// loaded G at a time and broadcast with shuffles; each nonzero streams one
// row of V, so consecutive lanes read consecutive 16-byte words.
// ---------------------------------------------------------------------------
template <typename T, int VEC>
struct VecIO;
template <typename T>
struct VecIO<T, 1> {
  static __device__ __forceinline__ void load(const T* p, T* v) { v[0] = p[0]; }
  static __device__ __forceinline__ void store(T* p, const T* v) { p[0] = v[0]; }
};
template <typename T>
struct VecIO<T, 2> {  // 2 x 8-byte elements
  static __device__ __forceinline__ void load(const T* p, T* v) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    memcpy(&v[0], &u.x, 8);
    memcpy(&v[1], &u.z, 8);
  }
  static __device__ __forceinline__ void store(T* p, const T* v) {
    uint4 u;
    memcpy(&u.x, &v[0], 8);
    memcpy(&u.z, &v[1], 8);
    *reinterpret_cast<uint4*>(p) = u;
  }
};
template <typename T>
struct VecIO<T, 4> {  // 4 x 4-byte elements
  static __device__ __forceinline__ void load(const T* p, T* v) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    memcpy(&v[0], &u.x, 4);
    memcpy(&v[1], &u.y, 4);
    memcpy(&v[2], &u.z, 4);
    memcpy(&v[3], &u.w, 4);
  }
  static __device__ __forceinline__ void store(T* p, const T* v) {
    uint4 u;
    memcpy(&u.x, &v[0], 4);
    memcpy(&u.y, &v[1], 4);
    memcpy(&u.z, &v[2], 4);
    memcpy(&u.w, &v[3], 4);
    *reinterpret_cast<uint4*>(p) = u;
  }
};

template <Arith A, int VEC, int G, int MAXT>
__global__ void __launch_bounds__(256) spmm_kernel(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const typename Pol<A>::T* __restrict__ val, int w, const typename Pol<A>::T* __restrict__ V,
    int64_t ldv, typename Pol<A>::T* __restrict__ Y, int64_t ldy, typename Pol<A>::S alpha,
    bool scale, typename Pol<A>::S beta, bool has_beta, const typename Pol<A>::T* __restrict__ U,
    int64_t ldu, typename Pol<A>::S gamma, bool has_gamma, int heavy_min) {
  using P = Pol<A>;
  using T = typename P::T;
  using S = typename P::S;
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  const int gbase = lane - g;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
  const int64_t group = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = int64_t(gridDim.x) * blockDim.x / G;

  for (int64_t row = group; row < n; row += ngroups) {
    typename P::Acc acc[MAXT][VEC];
#pragma unroll
    for (int t = 0; t < MAXT; ++t)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[t][v] = P::zero();
    const int start = rowptr[row], end = rowptr[row + 1];
    if (heavy_min > 0 && end - start > heavy_min) continue;  // spmm_heavy_kernel's row
    for (int base = start; base < end; base += G) {
      const int my = base + g;
      int cj = 0;
      S aj{};
      if (my < end) {
        cj = colind[my];
        T v = val[my];
        aj = scale ? scale_val<A>(v, alpha) : P::stage(v);
      }
      const int cnt = min(G, end - base);
      // UNR nonzeros per step: all their row loads are issued before the
      // multiply-adds, so a warp keeps several neighbour rows in flight
      constexpr int UNR = MAXT <= 4 ? 2 : 1;
      for (int t0 = 0; t0 < cnt; t0 += UNR) {
        const T* vrow[UNR];
        S a[UNR];
        bool ok[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int tt = min(t0 + u, cnt - 1);  // every lane of the group shuffles
          const int c = __shfl_sync(mask, cj, gbase + tt, 32);
          a[u] = shfl_t<S>(mask, aj, gbase + tt, 32);
          ok[u] = t0 + u < cnt;
          vrow[u] = V + int64_t(c) * ldv;
        }
        T x[UNR][MAXT][VEC];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int s = 0; s < MAXT; ++s) {
            const int col = (g + s * G) * VEC;
            if (ok[u] && col < w) {
              if (col + VEC <= w) {
                VecIO<T, VEC>::load(vrow[u] + col, x[u][s]);
              } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) x[u][s][v] = (col + v < w) ? vrow[u][col + v] : T{};
              }
            }
          }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int s = 0; s < MAXT; ++s) {
            const int col = (g + s * G) * VEC;
            if (ok[u] && col < w) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) P::mac(acc[s][v], a[u], P::stage(x[u][s][v]));
            }
          }
      }
    }
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
      const int col = (g + s * G) * VEC;
      if (col >= w) continue;
      if (has_beta || has_gamma) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          if (col + v >= w) continue;
          if (has_beta) P::mac(acc[s][v], beta, P::stage(V[row * ldv + col + v]));
          if (has_gamma) P::mac(acc[s][v], gamma, P::stage(U[row * ldu + col + v]));
        }
      }
      T out[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) out[v] = P::store(acc[s][v]);
      if (col + VEC <= w) {
        VecIO<T, VEC>::store(Y + row * ldy + col, out);
      } else {
        for (int v = 0; v < VEC && col + v < w; ++v) Y[row * ldy + col + v] = out[v];
      }
    }
  }
}

// Power-law rows: a row with more than heavy_min nonzeros would keep one lane
// group busy for its whole length while the rest of the grid idles.  Such
// rows (listed once per matrix) get one CTA each: warp q of HV (8, or fewer
// for wide rows) takes the row's nonzeros in blocks of 32 starting at block q
// (stride HV blocks),
// each lane its column vectors as in spmm_kernel; the HV partial rows are
// summed in warp order through shared memory (deterministic), then the
// epilogue of spmm_kernel.
__device__ __forceinline__ void acc_add(double& c, double x) { c += x; }
__device__ __forceinline__ void acc_add(float& c, float x) { c += x; }
__device__ __forceinline__ void acc_add(dd& c, dd x) {
  const float s = c.hi + x.hi;
  const float z = s - c.hi;
  const float t = (c.hi - (s - z)) + (x.hi - z);
  c.hi = s;
  c.lo += t + x.lo;
}

// warps per split row: 8, fewer when their partial rows would not fit in
// 48 KB of shared memory
template <Arith A, int VEC, int MAXT>
constexpr int hv_warps() {
  constexpr int per_warp = MAXT * VEC * 32 * int(sizeof(typename Pol<A>::Acc));
  return 49152 / per_warp < 8 ? 49152 / per_warp : 8;
}

template <Arith A, int VEC, int MAXT>
__global__ void __launch_bounds__(256) spmm_heavy_kernel(
    const int32_t* __restrict__ heavy, int nheavy, const int32_t* __restrict__ rowptr,
    const int32_t* __restrict__ colind, const typename Pol<A>::T* __restrict__ val, int w,
    const typename Pol<A>::T* __restrict__ V, int64_t ldv, typename Pol<A>::T* __restrict__ Y, int64_t ldy,
    typename Pol<A>::S alpha, bool scale, typename Pol<A>::S beta, bool has_beta,
    const typename Pol<A>::T* __restrict__ U, int64_t ldu, typename Pol<A>::S gamma, bool has_gamma) {
  using P = Pol<A>;
  using T = typename P::T;
  using S = typename P::S;
  using Acc = typename P::Acc;
  constexpr int G = 32;
  constexpr int HV_WARPS = hv_warps<A, VEC, MAXT>();
  __shared__ Acc red[HV_WARPS][MAXT * VEC][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int hrow = blockIdx.x; hrow < nheavy; hrow += gridDim.x) {
    const int64_t row = heavy[hrow];
    Acc acc[MAXT][VEC];
#pragma unroll
    for (int t = 0; t < MAXT; ++t)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[t][v] = P::zero();
    const int start = rowptr[row], end = rowptr[row + 1];
    for (int base = start + G * warp; base < end; base += G * HV_WARPS) {
      const int my = base + lane;
      int cj = 0;
      S aj{};
      if (my < end) {
        cj = colind[my];
        T v = val[my];
        aj = scale ? scale_val<A>(v, alpha) : P::stage(v);
      }
      const int cnt = min(G, end - base);
      for (int tt = 0; tt < cnt; ++tt) {
        const int c = __shfl_sync(0xffffffffu, cj, tt);
        const S a = shfl_t<S>(0xffffffffu, aj, tt, 32);
        const T* vrow = V + int64_t(c) * ldv;
#pragma unroll
        for (int s = 0; s < MAXT; ++s) {
          const int col = (lane + s * G) * VEC;
          if (col < w) {
            T x[VEC];
            if (col + VEC <= w) {
              VecIO<T, VEC>::load(vrow + col, x);
            } else {
#pragma unroll
              for (int v = 0; v < VEC; ++v) x[v] = (col + v < w) ? vrow[col + v] : T{};
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) P::mac(acc[s][v], a, P::stage(x[v]));
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < MAXT; ++s)
#pragma unroll
      for (int v = 0; v < VEC; ++v) red[warp][s * VEC + v][lane] = acc[s][v];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int s = 0; s < MAXT; ++s) {
        const int col = (lane + s * G) * VEC;
#pragma unroll
        for (int v = 0; v < VEC; ++v)
#pragma unroll
          for (int q = 1; q < HV_WARPS; ++q) acc_add(acc[s][v], red[q][s * VEC + v][lane]);
        if (col >= w) continue;
        if (has_beta || has_gamma) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (col + v >= w) continue;
            if (has_beta) P::mac(acc[s][v], beta, P::stage(V[row * ldv + col + v]));
            if (has_gamma) P::mac(acc[s][v], gamma, P::stage(U[row * ldu + col + v]));
          }
        }
        T out[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) out[v] = P::store(acc[s][v]);
        if (col + VEC <= w) {
          VecIO<T, VEC>::store(Y + row * ldy + col, out);
        } else {
          for (int v = 0; v < VEC && col + v < w; ++v) Y[row * ldy + col + v] = out[v];
        }
      }
    }
    __syncthreads();  // red is reused by the next row
  }
}

template <Arith A, int VEC, int G, int MAXT>
static void launch_spmm(const Csr<A>& M, int w, const typename Pol<A>::T* V, int64_t ldv,
                        typename Pol<A>::T* Y, int64_t ldy, double alpha, double beta,
                        const typename Pol<A>::T* U, int64_t ldu, double gamma, cudaStream_t st) {
  const int threads = 256;
  const int64_t rows_per_block = threads / G;
  int64_t blocks = cdiv(M.n, rows_per_block);
  const int64_t cap = int64_t(num_sms()) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const int hmin = (M.heavy && M.nheavy > 0) ? M.heavy_min : 0;
  spmm_kernel<A, VEC, G, MAXT><<<(unsigned)blocks, threads, 0, st>>>(
      M.n, M.rowptr, M.colind, M.val, w, V, ldv, Y, ldy, host_coef<A>(alpha), alpha != 1.0,
      host_coef<A>(beta), beta != 0.0, U, ldu, host_coef<A>(gamma), gamma != 0.0, hmin); count_launches(1);
  if (hmin > 0) {
    // the split rows need every lane of a warp per row: 32 lanes x VEC x
    // HMAXT column vectors cover the same columns as the G x MAXT of the
    // main kernel
    constexpr int HMAXT = (G * MAXT + 31) / 32;
    const int hb = M.nheavy < num_sms() * 8 ? M.nheavy : num_sms() * 8;
    spmm_heavy_kernel<A, VEC, HMAXT><<<(unsigned)hb, 32 * hv_warps<A, VEC, HMAXT>(), 0, st>>>(
        M.heavy, M.nheavy, M.rowptr, M.colind, M.val, w, V, ldv, Y, ldy, host_coef<A>(alpha), alpha != 1.0,
        host_coef<A>(beta), beta != 0.0, U, ldu, host_coef<A>(gamma), gamma != 0.0); count_launches(1);
  }
}

template <Arith A, int VEC>
static void spmm_dispatch_g(const Csr<A>& M, int w, const typename Pol<A>::T* V, int64_t ldv,
                            typename Pol<A>::T* Y, int64_t ldy, double alpha, double beta,
                            const typename Pol<A>::T* U, int64_t ldu, double gamma,
                            cudaStream_t st) {
  const int wv = (w + VEC - 1) / VEC;  // column vectors
  if (wv <= 4)
    launch_spmm<A, VEC, 4, 1>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 8)
    launch_spmm<A, VEC, 8, 1>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 16)
    launch_spmm<A, VEC, 16, 1>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 32)
    launch_spmm<A, VEC, 32, 1>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  // 3 and 6 vectors per lane for the widths between the powers of two (a
  // shrunk block of nes = k_max / 2 + 5 columns): a lane slot past the last
  // column still issues its loads and multiply-adds, predicated off
  else if (wv <= 48)
    launch_spmm<A, VEC, 16, 3>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 64)
    launch_spmm<A, VEC, 32, 2>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 96)
    launch_spmm<A, VEC, 32, 3>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 128)
    launch_spmm<A, VEC, 32, 4>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else if (wv <= 192)
    launch_spmm<A, VEC, 32, 6>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
  else
    launch_spmm<A, VEC, 32, 8>(M, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
}

template <Arith A>
cudaError_t spmm(const Csr<A>& M, int w, const typename Pol<A>::T* V, int64_t ldv,
                 typename Pol<A>::T* Y, int64_t ldy, double alpha, double beta,
                 const typename Pol<A>::T* U, int64_t ldu, double gamma, cudaStream_t st) {
  using T = typename Pol<A>::T;
  if (M.n <= 0 || w <= 0) return cudaSuccess;
  constexpr int VEC = 16 / sizeof(T);
  // column chunks of at most 256 vectors per launch
  const int chunk = 256 * VEC;
  for (int c0 = 0; c0 < w; c0 += chunk) {
    const int wc = (w - c0 < chunk) ? (w - c0) : chunk;
    const T* Vc = V + c0;
    T* Yc = Y + c0;
    const T* Uc = U ? U + c0 : nullptr;
    bool vec_ok = (ldv % VEC == 0) && (ldy % VEC == 0) &&
                  (reinterpret_cast<uintptr_t>(Vc) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(Yc) % 16 == 0);
    if (vec_ok)
      spmm_dispatch_g<A, VEC>(M, wc, Vc, ldv, Yc, ldy, alpha, beta, Uc, ldu, gamma, st);
    else
      spmm_dispatch_g<A, 1>(M, wc, Vc, ldv, Yc, ldy, alpha, beta, Uc, ldu, gamma, st);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K2: tall-skinny Gram G = U^T V, split-K over rows.
// CTA (tm, tn, z) computes the 64 x 64 tile (tm, tn) over row slice z into a
// float64 partial tile; gram_reduce sums the slices in a fixed order.
// 256 threads, 4 x 4 outputs per thread at (ty + 16 i, tx + 16 j).
// ---------------------------------------------------------------------------
constexpr int GT = 64;   // tile edge
constexpr int GK = 32;   // rows per shared-memory stage

template <Arith A>
__global__ void __launch_bounds__(256) gram_kernel(int64_t n, Blk<typename Pol<A>::T> U,
                                                   Blk<typename Pol<A>::T> V, bool sym,
                                                   int64_t rows_per_split, double* __restrict__ part,
                                                   const int* gate) {
  using P = Pol<A>;
  using T = typename P::T;
  using S = typename P::S;
  if (gate && *gate == 0) return;
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (sym && tm > tn) return;
  const int a = U.width, b = V.width;
  const int m0 = tm * GT, n0 = tn * GT;
  __shared__ S Us[GK][GT];
  __shared__ S Vs[GK][GT];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  // loader: fixed column per thread, rows t/64 + 4 i
  const int lc = t & 63, lr = t >> 6;
  const T* up = nullptr;
  int64_t uld = 0;
  const T* vp = nullptr;
  int64_t vld = 0;
  if (m0 + lc < a) {
    T* p;
    int s0;
    U.seg(m0 + lc, p, uld, s0);
    up = p + (m0 + lc - s0);
  }
  if (n0 + lc < b) {
    T* p;
    int s0;
    V.seg(n0 + lc, p, vld, s0);
    vp = p + (n0 + lc - s0);
  }
  typename P::Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = P::zero();

  const int64_t r_begin = int64_t(blockIdx.z) * rows_per_split;
  int64_t r_end = r_begin + rows_per_split;
  if (r_end > n) r_end = n;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GK) {
#pragma unroll
    for (int i = 0; i < GK / 4; ++i) {
      const int rr = lr + 4 * i;
      const int64_t r = r0 + rr;
      const bool rin = r < r_end;
      Us[rr][lc] = (up && rin) ? P::stage(up[r * uld]) : S{};
      Vs[rr][lc] = (vp && rin) ? P::stage(vp[r * vld]) : S{};
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      S av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Us[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Vs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) P::mac(acc[i][j], av[i], bv[j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) P::renorm(acc[i][j]);
    __syncthreads();
  }
  double* out = part + int64_t(blockIdx.z) * a * b;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= a) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c < b) out[int64_t(r) * b + c] = P::out(acc[i][j]);
    }
  }
}

__global__ void gram_reduce_kernel(int a, int b, int nsplit, bool sym, const double* __restrict__ part,
                                   double* __restrict__ G, int64_t ldg, const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(a) * b) return;
  int i = int(idx / b), j = int(idx % b);
  int si = i, sj = j;
  if (sym && i > j) {  // mirror the upper triangle: exact symmetry
    si = j;
    sj = i;
  }
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += part[int64_t(z) * a * b + int64_t(si) * b + sj];
  G[int64_t(i) * ldg + j] = s;
}

cudaError_t gram_reduce(int a, int b, int nsplit, bool sym, const double* part, double* G, int64_t ldg,
                        cudaStream_t st, const int* gate) {
  const int64_t tot = int64_t(a) * b;
  if (tot <= 0) return cudaSuccess;
  gram_reduce_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(a, b, nsplit, sym, part, G, ldg, gate);
  count_launches(1);
  return cudaGetLastError();
}

static int gram_nsplit(int64_t n, int a, int b, bool sym) {
  const int ta = (a + GT - 1) / GT, tb = (b + GT - 1) / GT;
  int tiles = sym ? (ta * (ta + 1)) / 2 : ta * tb;
  if (sym && ta != tb) tiles = ta * tb;
  int target = num_sms() * 4;
  int ns = (target + tiles - 1) / tiles;
  int64_t max_ns = cdiv(n, GK * 2);  // at least 64 rows per split (short inputs: more splits)
  if (ns > max_ns) ns = (int)max_ns;
  if (ns < 1) ns = 1;
  return ns;
}

size_t gram_scratch_elems(int64_t n, int a, int b, bool sym) {
  return size_t(gram_nsplit(n, a, b, sym)) * size_t(a) * size_t(b);
}

template <Arith A>
cudaError_t gram(int64_t n, const Blk<typename Pol<A>::T>& U, const Blk<typename Pol<A>::T>& V,
                 bool sym, double* G, int64_t ldg, double* scratch, cudaStream_t st,
                 const int* gate) {
  const int a = U.width, b = V.width;
  if (a <= 0 || b <= 0) return cudaSuccess;
  const int ns = gram_nsplit(n, a, b, sym);
  int64_t rps = cdiv(n, ns);
  rps = cdiv(rps, GK) * GK;
  dim3 grid((b + GT - 1) / GT, (a + GT - 1) / GT, ns);
  gram_kernel<A><<<grid, 256, 0, st>>>(n, U, V, sym, rps, scratch, gate); count_launches(1);
  const int64_t tot = int64_t(a) * b;
  gram_reduce_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(a, b, ns, sym, scratch, G, ldg, gate); count_launches(1);
  return cudaGetLastError();
}

// Same product with the split count capped so that the partial tiles fit in
// max_scratch_elems float64 elements (used by the allocation-free entry
// point, whose scratch has a fixed size).
template <Arith A>
cudaError_t gram_capped(int64_t n, const Blk<typename Pol<A>::T>& U, const Blk<typename Pol<A>::T>& V,
                        bool sym, double* G, int64_t ldg, double* scratch, size_t max_scratch_elems,
                        cudaStream_t st) {
  const int a = U.width, b = V.width;
  if (a <= 0 || b <= 0) return cudaSuccess;
  const size_t ab = size_t(a) * size_t(b);
  if (ab > max_scratch_elems) return cudaErrorInvalidValue;
  int ns = gram_nsplit(n, a, b, sym);
  const size_t cap = max_scratch_elems / ab;
  if (size_t(ns) > cap) ns = int(cap);
  int64_t rps = cdiv(n, ns);
  rps = cdiv(rps, GK) * GK;
  dim3 grid((b + GT - 1) / GT, (a + GT - 1) / GT, ns);
  gram_kernel<A><<<grid, 256, 0, st>>>(n, U, V, sym, rps, scratch, nullptr); count_launches(1);
  const int64_t tot = int64_t(a) * b;
  gram_reduce_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(a, b, ns, sym, scratch, G, ldg, nullptr); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K3: block update Y = U C + beta Y (row-streaming GEMM, C staged).
// CTA (tn, tm) computes rows [64 tm, 64 tm + 64) x columns [64 tn, ...);
// the column tile is the fast grid index so CTAs sharing U rows run together
// and U is read from HBM about once.
// ---------------------------------------------------------------------------
template <Arith A>
__global__ void __launch_bounds__(256) update_kernel(int64_t n, Blk<typename Pol<A>::T> U,
                                                     const typename Pol<A>::S* __restrict__ Cs,
                                                     int c, Blk<typename Pol<A>::T> Y,
                                                     typename Pol<A>::S beta, bool has_beta,
                                                     const int* gate) {
  using P = Pol<A>;
  using T = typename P::T;
  using S = typename P::S;
  if (gate && *gate == 0) return;
  const int s_dim = U.width;
  const int64_t m0 = int64_t(blockIdx.y) * GT;
  const int n0 = blockIdx.x * GT;
  __shared__ S Us[GK][GT + 1];
  __shared__ S Cs_[GK][GT];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int lk = t & 31, lr = t >> 5;  // U loader: k fastest, rows lr + 8 i
  typename P::Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = P::zero();

  for (int k0 = 0; k0 < s_dim; k0 += GK) {
    const int kk = k0 + lk;
    const T* up = nullptr;
    int64_t uld = 0;
    if (kk < s_dim) {
      T* p;
      int s0;
      U.seg(kk, p, uld, s0);
      up = p + (kk - s0);
    }
#pragma unroll
    for (int i = 0; i < GT / 8; ++i) {
      const int rr = lr + 8 * i;
      const int64_t r = m0 + rr;
      Us[lk][rr] = (up && r < n) ? P::stage(up[r * uld]) : S{};
    }
#pragma unroll
    for (int i = 0; i < (GK * GT) / 256; ++i) {
      const int idx = t + 256 * i;
      const int k = idx / GT, cc = idx % GT;
      Cs_[k][cc] = (k0 + k < s_dim && n0 + cc < c) ? Cs[int64_t(k0 + k) * c + n0 + cc] : S{};
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      S av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Us[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Cs_[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) P::mac(acc[i][j], av[i], bv[j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) P::renorm(acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = m0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = n0 + tx + 16 * j;
      if (cc >= c) continue;
      T* yp = Y.at(r, cc);
      if (has_beta) P::mac(acc[i][j], beta, P::stage(*yp));
      *yp = P::store(acc[i][j]);
    }
  }
}

template <Arith A>
__global__ void stage_coef_kernel(int s, int c, const double* __restrict__ C, int64_t ldc,
                                  typename Pol<A>::S* __restrict__ Cs, int64_t ldo, double scale,
                                  const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(s) * c) return;
  const int i = int(idx / c), j = int(idx % c);
  Cs[int64_t(i) * ldo + j] = Pol<A>::stage_coef(scale * C[int64_t(i) * ldc + j]);
}

template <Arith A>
cudaError_t stage_coef(int s, int c, const double* C, int64_t ldc, typename Pol<A>::S* Cs,
                       int64_t ldo, double scale, cudaStream_t st, const int* gate) {
  const int64_t tot = int64_t(s) * c;
  if (tot <= 0) return cudaSuccess;
  stage_coef_kernel<A><<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(s, c, C, ldc, Cs, ldo, scale, gate); count_launches(1);
  return cudaGetLastError();
}

// Y = a U + b V elementwise over an n x w view (Y may alias U or V).
template <Arith A>
__global__ void axpby_kernel(int64_t n, int w, const typename Pol<A>::T* U, int64_t ldu,
                             typename Pol<A>::S a, const typename Pol<A>::T* V, int64_t ldv,
                             typename Pol<A>::S b, typename Pol<A>::T* Y, int64_t ldy) {
  using P = Pol<A>;
  const int64_t tot = n * w;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = idx / w;
    const int c = int(idx % w);
    typename P::Acc acc = P::zero();
    P::mac(acc, a, P::stage(U[r * ldu + c]));
    P::mac(acc, b, P::stage(V[r * ldv + c]));
    Y[r * ldy + c] = P::store(acc);
  }
}

template <Arith A>
cudaError_t axpby(int64_t n, int w, const typename Pol<A>::T* U, int64_t ldu, double a,
                  const typename Pol<A>::T* V, int64_t ldv, double b, typename Pol<A>::T* Y,
                  int64_t ldy, cudaStream_t st) {
  const int64_t tot = n * w;
  if (tot <= 0) return cudaSuccess;
  int64_t blocks = cdiv(tot, 256);
  const int64_t cap = int64_t(num_sms()) * 16;
  if (blocks > cap) blocks = cap;
  axpby_kernel<A><<<(unsigned)blocks, 256, 0, st>>>(n, w, U, ldu, host_coef<A>(a), V, ldv,
                                                    host_coef<A>(b), Y, ldy); count_launches(1);
  return cudaGetLastError();
}

// gated 2D copy (used for the conditional third CholeskyQR pass)
template <typename T>
__global__ void copy_blk_kernel(int64_t n, Blk<T> src, Blk<T> dst, const int* gate) {
  if (gate && *gate == 0) return;
  const int w = src.width;
  const int64_t tot = n * w;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = idx / w;
    const int c = int(idx % w);
    *dst.at(r, c) = *src.at(r, c);
  }
}

template <typename T>
cudaError_t copy_blk(int64_t n, const Blk<T>& src, const Blk<T>& dst, cudaStream_t st, const int* gate) {
  const int64_t tot = n * src.width;
  if (tot <= 0) return cudaSuccess;
  int64_t blocks = cdiv(tot, 256);
  const int64_t cap = int64_t(num_sms()) * 16;
  if (blocks > cap) blocks = cap;
  copy_blk_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(n, src, dst, gate); count_launches(1);
  return cudaGetLastError();
}
template cudaError_t copy_blk<double>(int64_t, const Blk<double>&, const Blk<double>&, cudaStream_t, const int*);
template cudaError_t copy_blk<dd>(int64_t, const Blk<dd>&, const Blk<dd>&, cudaStream_t, const int*);
template cudaError_t copy_blk<float>(int64_t, const Blk<float>&, const Blk<float>&, cudaStream_t, const int*);

template <Arith A>
cudaError_t update(int64_t n, const Blk<typename Pol<A>::T>& U, const typename Pol<A>::S* Cs,
                   int c, const Blk<typename Pol<A>::T>& Y, double beta, cudaStream_t st,
                   const int* gate) {
  if (n <= 0 || c <= 0) return cudaSuccess;
  dim3 grid((c + GT - 1) / GT, (unsigned)cdiv(n, GT));
  update_kernel<A><<<grid, 256, 0, st>>>(n, U, Cs, c, Y, host_coef<A>(beta), beta != 0.0, gate); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4: residual R = T (AX - X diag(lam)), squared column norms of X and of the
// unpreconditioned residual.  Block (32, 8): tx walks 32 consecutive columns,
// ty rows; per-block partial norms go to scratch and are summed in a fixed
// order by residual_reduce.
// ---------------------------------------------------------------------------
constexpr int RES_ROWS = 8;

static int residual_blocks(int64_t n) {
  int64_t b = cdiv(n, 256);
  const int64_t cap = int64_t(num_sms()) * 4;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

size_t residual_scratch_elems(int64_t n, int w) { return size_t(2) * residual_blocks(n) * size_t(w); }

template <Arith A>
__global__ void __launch_bounds__(256) residual_kernel(
    int64_t n, int w, const typename Pol<A>::T* __restrict__ X, int64_t ldx,
    const typename Pol<A>::T* __restrict__ AX, int64_t ldax, const double* __restrict__ lam,
    const typename Pol<A>::T* __restrict__ tdiag, typename Pol<A>::T* __restrict__ R, int64_t ldr,
    int64_t rows_per_block, double* __restrict__ part) {
  using P = Pol<A>;
  using T = typename P::T;
  using S = typename P::S;
  __shared__ double red[2][RES_ROWS][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t r_begin = int64_t(blockIdx.x) * rows_per_block;
  int64_t r_end = r_begin + rows_per_block;
  if (r_end > n) r_end = n;
  for (int c0 = 0; c0 < w; c0 += 32) {
    const int c = c0 + tx;
    typename P::Acc xn = P::zero(), rn = P::zero();
    if (c < w) {
      const S nl = P::stage_coef(-lam[c]);
      for (int64_t r = r_begin + ty; r < r_end; r += RES_ROWS) {
        const T x = X[r * ldx + c];
        typename P::Acc acc = acc_from<A>(AX[r * ldax + c]);
        P::mac(acc, nl, P::stage(x));
        const T rv = P::store(acc);
        P::mac(xn, P::stage(x), P::stage(x));
        P::mac(rn, P::stage(rv), P::stage(rv));
        if (R) {
          if (tdiag) {
            typename P::Acc o = P::zero();
            P::mac(o, P::stage(tdiag[r]), P::stage(rv));
            R[r * ldr + c] = P::store(o);
          } else {
            R[r * ldr + c] = rv;
          }
        }
      }
    }
    red[0][ty][tx] = P::out(xn);
    red[1][ty][tx] = P::out(rn);
    __syncthreads();
    if (ty == 0 && c < w) {
      double sx = 0.0, sr = 0.0;
      for (int i = 0; i < RES_ROWS; ++i) {
        sx += red[0][i][tx];
        sr += red[1][i][tx];
      }
      part[(int64_t(blockIdx.x) * 2 + 0) * w + c] = sx;
      part[(int64_t(blockIdx.x) * 2 + 1) * w + c] = sr;
    }
    __syncthreads();
  }
}

__global__ void residual_reduce_kernel(int w, int nblocks, const double* __restrict__ part,
                                       double* __restrict__ xnorm2, double* __restrict__ rnorm2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w) return;
  double sx = 0.0, sr = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    sx += part[(int64_t(b) * 2 + 0) * w + c];
    sr += part[(int64_t(b) * 2 + 1) * w + c];
  }
  if (xnorm2) xnorm2[c] = sx;
  if (rnorm2) rnorm2[c] = sr;
}

template <Arith A>
cudaError_t residual(int64_t n, int w, const typename Pol<A>::T* X, int64_t ldx,
                     const typename Pol<A>::T* AX, int64_t ldax, const double* lam,
                     const typename Pol<A>::T* tdiag, typename Pol<A>::T* R, int64_t ldr,
                     double* xnorm2, double* rnorm2, double* scratch, cudaStream_t st) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  const int nb = residual_blocks(n);
  const int64_t rpb = cdiv(n, nb);
  residual_kernel<A><<<nb, dim3(32, RES_ROWS), 0, st>>>(n, w, X, ldx, AX, ldax, lam, tdiag, R, ldr,
                                                        rpb, scratch); count_launches(1);
  residual_reduce_kernel<<<(w + 127) / 128, 128, 0, st>>>(w, nb, scratch, xnorm2, rnorm2); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// format conversion (float64 <-> float32 <-> double-float)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_as_double(const void* p, int dt, int64_t i) {
  if (dt == EIG_F64) return static_cast<const double*>(p)[i];
  if (dt == EIG_F32) return (double)static_cast<const float*>(p)[i];
  dd v = static_cast<const dd*>(p)[i];
  return dd_to_double(v);
}
__device__ __forceinline__ void store_from_double(void* p, int dt, int64_t i, double x) {
  if (dt == EIG_F64)
    static_cast<double*>(p)[i] = x;
  else if (dt == EIG_F32)
    static_cast<float*>(p)[i] = (float)x;
  else
    static_cast<dd*>(p)[i] = dd_split(x);
}

__global__ void convert2d_kernel(int64_t rows, int64_t cols, const void* src, int64_t lds, int sdt,
                                 void* dst, int64_t ldd, int ddt) {
  const int64_t tot = rows * cols;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = idx / cols, c = idx % cols;
    store_from_double(dst, ddt, r * ldd + c, load_as_double(src, sdt, r * lds + c));
  }
}

cudaError_t convert2d(int64_t rows, int64_t cols, const void* src, int64_t lds, int sdt, void* dst,
                      int64_t ldd, int ddt, cudaStream_t st) {
  const int64_t tot = rows * cols;
  if (tot <= 0) return cudaSuccess;
  int64_t blocks = cdiv(tot, 256);
  const int64_t cap = int64_t(num_sms()) * 32;
  if (blocks > cap) blocks = cap;
  convert2d_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, cols, src, lds, sdt, dst, ldd, ddt); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gaussian columns of the 'Random' expansion (Sec. 6.4), drawn from a
// counter-based generator so that every entry is a function of (seed,
// expansion e, row i, column j): Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// SC'11; multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key increments
// 0x9E3779B9 and 0xBB67AE85, ten rounds) on the counter
// (i mod 2^32, i / 2^32, j / 2, e) with key (seed mod 2^32, seed / 2^32);
// its words give two float64 uniforms u1 = (w0 2^21 + w1 / 2^11 + 1/2) 2^-53
// in (0, 1) and u2 = (w2 2^21 + w3 / 2^11) 2^-53, and Box-Muller gives
// sqrt(-2 ln u1) times cos(2 pi u2) (even j) or sin(2 pi u2) (odd j).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__global__ void gauss_fill_kernel(int64_t n, int w, void* dst, int64_t ld, int dt, uint64_t seed, uint32_t e) {
  const int64_t tot = n * w;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = idx / w;
    const int j = int(idx % w);
    uint32_t c[4] = {uint32_t(uint64_t(i)), uint32_t(uint64_t(i) >> 32), uint32_t(j >> 1), e};
    philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
    const double u1 = (double(c[0]) * 2097152.0 + double(c[1] >> 11) + 0.5) * 0x1p-53;
    const double u2 = (double(c[2]) * 2097152.0 + double(c[3] >> 11)) * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    const double ang = 6.283185307179586 * u2;  // 2 pi rounded to float64, as 2.0 * pi
    store_from_double(dst, dt, i * ld + j, (j & 1) ? r * sin(ang) : r * cos(ang));
  }
}

cudaError_t gauss_fill(int64_t n, int w, void* dst, int64_t ld, int dt, uint64_t seed, int e, cudaStream_t st) {
  const int64_t tot = n * w;
  if (tot <= 0) return cudaSuccess;
  int64_t blocks = cdiv(tot, 256);
  const int64_t cap = int64_t(num_sms()) * 32;
  if (blocks > cap) blocks = cap;
  gauss_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, w, dst, ld, dt, seed, uint32_t(e)); count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define EIG_INST(A)                                                                               \
  template cudaError_t spmm<A>(const Csr<A>&, int, const Pol<A>::T*, int64_t, Pol<A>::T*, int64_t, \
                               double, double, const Pol<A>::T*, int64_t, double, cudaStream_t);  \
  template cudaError_t gram<A>(int64_t, const Blk<Pol<A>::T>&, const Blk<Pol<A>::T>&, bool,       \
                               double*, int64_t, double*, cudaStream_t, const int*);              \
  template cudaError_t stage_coef<A>(int, int, const double*, int64_t, Pol<A>::S*, int64_t,       \
                                     double, cudaStream_t, const int*);                           \
  template cudaError_t axpby<A>(int64_t, int, const Pol<A>::T*, int64_t, double, const Pol<A>::T*, \
                                int64_t, double, Pol<A>::T*, int64_t, cudaStream_t);              \
  template cudaError_t update<A>(int64_t, const Blk<Pol<A>::T>&, const Pol<A>::S*, int,           \
                                 const Blk<Pol<A>::T>&, double, cudaStream_t, const int*);        \
  template cudaError_t residual<A>(int64_t, int, const Pol<A>::T*, int64_t, const Pol<A>::T*,     \
                                   int64_t, const double*, const Pol<A>::T*, Pol<A>::T*, int64_t, \
                                   double*, double*, double*, cudaStream_t);

EIG_INST(Arith::F64)
EIG_INST(Arith::DF64)
EIG_INST(Arith::F32)
EIG_INST(Arith::C32)

#define EIG_INST_CAPPED(A)                                                                          \
  template cudaError_t gram_capped<A>(int64_t, const Blk<Pol<A>::T>&, const Blk<Pol<A>::T>&, bool, \
                                      double*, int64_t, double*, size_t, cudaStream_t);
EIG_INST_CAPPED(Arith::F64)
EIG_INST_CAPPED(Arith::DF64)
EIG_INST_CAPPED(Arith::F32)
EIG_INST_CAPPED(Arith::C32)

}  // namespace eig
