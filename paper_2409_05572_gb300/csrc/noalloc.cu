// Allocation-free Gram product (eig_gram_noalloc in include/eig_gb300.h).
//
// eig_gram takes its split-K scratch from cudaMallocAsync on every call.
// Some callers cannot allocate device memory on their call path: a serving
// process that has handed all of HBM to its own pool at start-up, or host
// code that runs where a cudaMalloc/cudaFree (which may synchronise the
// device or fail under memory pressure) is not allowed.  This variant uses a
// fixed scratch array that lives in this file's module instead.
//
// The scratch is a file-scope __device__ array of EIG_NOALLOC_SCRATCH_DOUBLES
// float64 elements (16 MiB).  Every GPU that loads the library keeps it until
// the process exits.  All calls share it: two calls whose kernels overlap on
// the GPU (different streams without ordering, or different host threads)
// race on it.  Nothing in it has to start at zero: every partial tile the
// reduction reads is written by the same call first.
#include <cstdio>
#include <mutex>

#include "blocks.cuh"

using namespace eig;

static __device__ __align__(256) double g_gram_scratch[EIG_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device, looked up once per
// device.  The host-side name g_gram_scratch is only a stand-in for the
// symbol and must never be passed to a kernel.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EIG_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess || p == nullptr) return EIG_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return EIG_OK;
}

template <Arith A>
int gram_noalloc_t(int64_t n, int a, int b, const void* U, int64_t ldu, const void* V, int64_t ldv, int sym,
                   double* G, int64_t ldg, cudaStream_t st) {
  using T = typename Pol<A>::T;
  double* scr = nullptr;
  int rc = scratch_address(&scr);
  if (rc) return rc;
  Blk<T> Ub, Vb;
  Ub.add(static_cast<T*>(const_cast<void*>(U)), ldu, a);
  Vb.add(static_cast<T*>(const_cast<void*>(V)), ldv, b);
  cudaError_t e = gram_capped<A>(n, Ub, Vb, sym != 0, G, ldg, scr, EIG_NOALLOC_SCRATCH_DOUBLES, st);
  return e == cudaSuccess ? EIG_OK : EIG_ECUDA;
}

}  // namespace

extern "C" int eig_gram_noalloc(int64_t n, int a, int b, const void* U, int64_t ldu, const void* V, int64_t ldv,
                                int arith, int sym, double* G, int64_t ldg, void* stream) {
  if (n < 0 || a < 0 || b < 0 || ldu < a || ldv < b || ldg < b) return EIG_EINVAL;
  if (arith < EIG_ARITH_F64 || arith > EIG_ARITH_C32 || (sym && a != b)) return EIG_EINVAL;
  if (a == 0 || b == 0) return EIG_OK;
  if (int64_t(a) * int64_t(b) > int64_t(EIG_NOALLOC_SCRATCH_DOUBLES)) return EIG_EINVAL;
  if (!U || !V || !G) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    return cudaMemset2DAsync(G, sizeof(double) * ldg, 0, sizeof(double) * b, a, st) == cudaSuccess ? EIG_OK
                                                                                                  : EIG_ECUDA;
  }
  switch (arith) {
    case EIG_ARITH_F64: return gram_noalloc_t<Arith::F64>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_DF64: return gram_noalloc_t<Arith::DF64>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_F32: return gram_noalloc_t<Arith::F32>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    default: return gram_noalloc_t<Arith::C32>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
  }
}
