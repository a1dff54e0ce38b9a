// Shared device-side definitions of the GB300 eigensolver library:
// block descriptors, the four arithmetic policies and small helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/eig_gb300.h"

namespace eig {

// ---------------------------------------------------------------------------
// A logical n x w block made of up to MAX_SEG column segments.  Segment t is
// a row-major n x w_t view starting at ptr with leading dimension ld
// (elements).  Logical column c maps to the segment holding it.  Every block
// of the method (X, P, W, S = [X, P, W], S_drop halves) is such a view, so
// widths change without copies.
// ---------------------------------------------------------------------------
constexpr int MAX_SEG = 4;

template <typename T>
struct Blk {
  int nseg = 0;
  int width = 0;
  T* ptr[MAX_SEG] = {nullptr, nullptr, nullptr, nullptr};
  int64_t ld[MAX_SEG] = {0, 0, 0, 0};
  int start[MAX_SEG + 1] = {0, 0, 0, 0, 0};  // logical first column of segment t

  __host__ __device__ void add(T* p, int64_t l, int w) {
    if (w <= 0) return;
    ptr[nseg] = p;
    ld[nseg] = l;
    start[nseg] = width;
    width += w;
    start[nseg + 1] = width;
    ++nseg;
  }
  // segment of logical column c (c < width): its pointer, leading dimension
  // and first logical column, by unrolled selects, so that a kernel reading a
  // Blk parameter never indexes it dynamically (which would copy the
  // parameter to local memory)
  __host__ __device__ __forceinline__ void seg(int c, T*& p, int64_t& l, int& s0) const {
    p = ptr[0];
    l = ld[0];
    s0 = start[0];
#pragma unroll
    for (int t = 1; t < MAX_SEG; ++t)
      if (t < nseg && c >= start[t]) {
        p = ptr[t];
        l = ld[t];
        s0 = start[t];
      }
  }
  // address of element (row, logical column c); c < width
  __host__ __device__ T* at(int64_t row, int c) const {
    T* p;
    int64_t l;
    int s0;
    seg(c, p, l, s0);
    return p + row * l + (c - s0);
  }
};

// ---------------------------------------------------------------------------
// Arithmetic policies.
//   F64  : float64 storage, native FP64 FMA (1 TFLOP/s class on GB300).
//   DF64 : double-float storage {hi, lo} (value hi + lo) and arithmetic on
//          the FP32 pipes: a product is TwoProd(a_hi, b_hi) + a_hi b_lo +
//          a_lo b_hi (Dekker 1971) and sums are TwoSum-accumulated (Knuth)
//          with periodic renormalisation; about 2^-48 relative per operation.
//          GB300 runs FP64 at 1/72 of the FP32 rate, so the FP64 form keeps
//          every n-sized block in this format and touches no FP64 unit in its
//          n-sized loops.
//   F32  : float32 storage and arithmetic.
//   C32  : float32 storage, compensated dot products (Ogita, Rump and Oishi
//          2005, Dot2): TwoProd gives each product exactly, TwoSum keeps the
//          rounding error of the running sum.
// ---------------------------------------------------------------------------
struct __align__(8) dd { float hi, lo; };

__device__ __forceinline__ dd dd_split(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// acc += a * b (both split); lazy low part
__device__ __forceinline__ void dd_mac(dd& acc, dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s = acc.hi + p;
  float z = s - acc.hi;
  float t = (acc.hi - (s - z)) + (p - z);
  acc.hi = s;
  acc.lo += t + e;
}
// acc += a * b for plain floats, products exact (Dot2 step)
__device__ __forceinline__ void c32_mac(dd& acc, float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  float s = acc.hi + p;
  float z = s - acc.hi;
  float t = (acc.hi - (s - z)) + (p - z);
  acc.hi = s;
  acc.lo += t + e;
}
__device__ __forceinline__ void dd_renorm(dd& a) {
  float s = a.hi + a.lo;
  a.lo = a.lo - (s - a.hi);
  a.hi = s;
}

enum class Arith : int { F64 = 0, DF64 = 1, F32 = 2, C32 = 3 };

template <Arith A> struct Pol;

template <> struct Pol<Arith::F64> {
  using T = double;     // storage
  using S = double;     // staged (shared memory) operand
  using Acc = double;   // accumulator
  static __device__ __forceinline__ S stage(T x) { return x; }
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ void mac(Acc& c, S a, S b) { c = fma(a, b, c); }
  static __device__ __forceinline__ void renorm(Acc&) {}
  static __device__ __forceinline__ double out(Acc c) { return c; }
  static __device__ __forceinline__ S stage_coef(double x) { return x; }
  static __device__ __forceinline__ T store(Acc c) { return c; }
};
template <> struct Pol<Arith::DF64> {
  using T = dd;         // blocks are stored as double-float pairs
  using S = dd;
  using Acc = dd;
  static __device__ __forceinline__ S stage(T x) { return x; }
  static __device__ __forceinline__ Acc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void mac(Acc& c, S a, S b) { dd_mac(c, a, b); }
  static __device__ __forceinline__ void renorm(Acc& c) { dd_renorm(c); }
  static __device__ __forceinline__ double out(Acc c) { return dd_to_double(c); }
  static __device__ __forceinline__ S stage_coef(double x) { return dd_split(x); }
  static __device__ __forceinline__ T store(Acc c) { dd_renorm(c); return c; }
};
template <> struct Pol<Arith::F32> {
  using T = float;
  using S = float;
  using Acc = float;
  static __device__ __forceinline__ S stage(T x) { return x; }
  static __device__ __forceinline__ Acc zero() { return 0.f; }
  static __device__ __forceinline__ void mac(Acc& c, S a, S b) { c = fmaf(a, b, c); }
  static __device__ __forceinline__ void renorm(Acc&) {}
  static __device__ __forceinline__ double out(Acc c) { return (double)c; }
  static __device__ __forceinline__ S stage_coef(double x) { return (float)x; }
  static __device__ __forceinline__ T store(Acc c) { return c; }
};
template <> struct Pol<Arith::C32> {
  using T = float;
  using S = float;
  using Acc = dd;
  static __device__ __forceinline__ S stage(T x) { return x; }
  static __device__ __forceinline__ Acc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void mac(Acc& c, S a, S b) { c32_mac(c, a, b); }
  static __device__ __forceinline__ void renorm(Acc& c) { dd_renorm(c); }
  static __device__ __forceinline__ double out(Acc c) { return dd_to_double(c); }
  static __device__ __forceinline__ S stage_coef(double x) { return (float)x; }
  static __device__ __forceinline__ T store(Acc c) { return c.hi + c.lo; }
};

template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return (float)x; }

inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Host-side count of this library's kernel launches (all threads, all
// devices); eig_solve reports the difference over a solve.
void count_launches(int n);
int64_t launches_total();

}  // namespace eig
