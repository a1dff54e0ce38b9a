// Low-level C ABI entry points (include/eig_gb300.h): one call per step of
// the hot path, dispatched on element format / arithmetic.  Temporary device
// memory comes from cudaMallocAsync on the caller's stream.
#include <cstdio>
#include <type_traits>

#include "blocks.cuh"
#include "small.cuh"
#include "tc.cuh"

using namespace eig;

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? EIG_OK : EIG_ECUDA; }

// stream-ordered temporary allocation freed at scope exit
struct Tmp {
  void* p = nullptr;
  cudaStream_t st;
  explicit Tmp(cudaStream_t s) : st(s) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes > 0 ? bytes : 16, st); }
  ~Tmp() {
    if (p) cudaFreeAsync(p, st);
  }
};

template <typename T>
Blk<T> one(const void* p, int64_t ld, int w) {
  Blk<T> b;
  b.add(static_cast<T*>(const_cast<void*>(p)), ld, w);
  return b;
}

bool arith_ok(int a) { return a >= EIG_ARITH_F64 && a <= EIG_ARITH_C32; }
bool arith_tc(int a) { return a == EIG_ARITH_DF64_TC || a == EIG_ARITH_F64_TC; }

template <Arith A>
int gram_t(int64_t n, int a, int b, const void* U, int64_t ldu, const void* V, int64_t ldv, int sym,
           double* G, int64_t ldg, cudaStream_t st) {
  using T = typename Pol<A>::T;
  Tmp scr(st);
  if (scr.alloc(sizeof(double) * gram_scratch_elems(n, a, b, sym != 0)) != cudaSuccess) return EIG_ENOMEM;
  return cuda_status(gram<A>(n, one<T>(U, ldu, a), one<T>(V, ldv, b), sym != 0, G, ldg,
                             static_cast<double*>(scr.p), st));
}

template <Arith A>
int update_t(int64_t n, int s, int c, const void* U, int64_t ldu, const double* C, int64_t ldc, void* Y,
             int64_t ldy, double beta, cudaStream_t st) {
  using T = typename Pol<A>::T;
  using S = typename Pol<A>::S;
  Tmp cs(st);
  if (cs.alloc(sizeof(S) * size_t(s) * c) != cudaSuccess) return EIG_ENOMEM;
  cudaError_t e = stage_coef<A>(s, c, C, ldc, static_cast<S*>(cs.p), c, 1.0, st);
  if (e != cudaSuccess) return EIG_ECUDA;
  return cuda_status(update<A>(n, one<T>(U, ldu, s), static_cast<S*>(cs.p), c, one<T>(Y, ldy, c), beta, st));
}

// products on the tensor cores (k_tc.cu): T = dd (6 slices) or double (7)
template <typename T>
int gram_tc_t(int64_t n, int a, int b, const void* U, int64_t ldu, const void* V, int64_t ldv, int sym, double* G,
              int64_t ldg, cudaStream_t st) {
  const int ns = std::is_same<T, dd>::value ? tc::NS_DF : tc::NS_F64;
  const bool same = U == V && ldu == ldv && a == b;
  const size_t su = (tc_slice_bytes(ns, n, a) + 255) / 256 * 256;
  const size_t sv = same ? 0 : tc_slice_bytes(ns, n, b);
  Tmp sl(st), scr(st);
  if (sl.alloc(su + sv) != cudaSuccess) return EIG_ENOMEM;
  if (scr.alloc(sizeof(double) * gram_tc_scratch_elems(ns, n, a, b, sym != 0)) != cudaSuccess) return EIG_ENOMEM;
  char* pu = static_cast<char*>(sl.p);
  char* pv = same ? pu : pu + su;
  cudaError_t e = tc_slice_cols<T>(n, one<T>(U, ldu, a), pu, st);
  if (e == cudaSuccess && !same) e = tc_slice_cols<T>(n, one<T>(V, ldv, b), pv, st);
  if (e == cudaSuccess)
    e = gram_tc_product(ns, n, a, b, pu, pv, sym != 0, G, ldg, static_cast<double*>(scr.p), st);
  return cuda_status(e);
}

template <typename T>
int update_tc_t(int64_t n, int s, int c, const void* U, int64_t ldu, const double* C, int64_t ldc, void* Y,
                int64_t ldy, double beta, cudaStream_t st) {
  const int ns = std::is_same<T, dd>::value ? tc::NS_DF : tc::NS_F64;
  if (s == 0) {
    if (std::is_same<T, dd>::value) return update_t<Arith::DF64>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    return update_t<Arith::F64>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
  }
  const size_t su = (tc_slice_bytes(ns, s, n) + 255) / 256 * 256;
  Tmp sl(st);
  if (sl.alloc(su + tc_slice_bytes(ns, s, c)) != cudaSuccess) return EIG_ENOMEM;
  char* pu = static_cast<char*>(sl.p);
  char* pc = pu + su;
  cudaError_t e = tc_slice_coef(ns, s, c, C, ldc, 1.0, pc, st);
  if (e == cudaSuccess) e = tc_slice_rows<T>(n, one<T>(U, ldu, s), pu, st);
  if (e == cudaSuccess) e = update_tc_product<T>(n, s, c, pu, pc, one<T>(Y, ldy, c), beta, st);
  return cuda_status(e);
}

template <Arith A>
int residual_t(int64_t n, int w, const void* X, int64_t ldx, const void* AX, int64_t ldax, const double* lam,
               const void* tdiag, void* R, int64_t ldr, double* xn, double* rn, cudaStream_t st) {
  using T = typename Pol<A>::T;
  Tmp scr(st);
  if (scr.alloc(sizeof(double) * residual_scratch_elems(n, w)) != cudaSuccess) return EIG_ENOMEM;
  return cuda_status(residual<A>(n, w, static_cast<const T*>(X), ldx, static_cast<const T*>(AX), ldax, lam,
                                 static_cast<const T*>(tdiag), static_cast<T*>(R), ldr, xn, rn,
                                 static_cast<double*>(scr.p), st));
}

template <Arith A>
int spmm_t(int64_t n, const int32_t* rowptr, const int32_t* colind, const void* val, int w, const void* V,
           int64_t ldv, void* Y, int64_t ldy, double alpha, double beta, const void* U, int64_t ldu, double gamma,
           cudaStream_t st) {
  using T = typename Pol<A>::T;
  Csr<A> c;
  c.n = n;
  c.rowptr = rowptr;
  c.colind = colind;
  c.val = static_cast<const T*>(val);
  return cuda_status(spmm<A>(c, w, static_cast<const T*>(V), ldv, static_cast<T*>(Y), ldy, alpha, beta,
                             static_cast<const T*>(U), ldu, gamma, st));
}

template <Arith A>
int cholqr2_t(int64_t n, int w, void* W, int64_t ldw, int* status_out, cudaStream_t st) {
  using T = typename Pol<A>::T;
  using S = typename Pol<A>::S;
  const size_t esz = sizeof(T);
  Tmp scr(st), G(st), Rinv(st), work(st), Cs(st), tmp(st), flags(st);
  if (scr.alloc(sizeof(double) * gram_scratch_elems(n, w, w, true)) || G.alloc(sizeof(double) * w * w) ||
      Rinv.alloc(sizeof(double) * w * w) || work.alloc(sizeof(double) * (size_t(w) * w + 2 * size_t(w))) ||
      Cs.alloc(sizeof(S) * w * w) || tmp.alloc(esz * size_t(n) * w) || flags.alloc(sizeof(int) * 4))
    return EIG_ENOMEM;
  int* fl = static_cast<int*>(flags.p);
  if (cudaMemsetAsync(fl, 0, sizeof(int) * 4, st)) return EIG_ECUDA;
  Blk<T> Wb = one<T>(W, ldw, w);
  Blk<T> Tb = one<T>(tmp.p, w, w);
  // pass: G = W^T W, R^{-1}, dst = src R^{-1}
  auto pass = [&](const Blk<T>& src, const Blk<T>& dst, int slot, const int* gate) -> int {
    if (gram<A>(n, src, src, true, static_cast<double*>(G.p), w, static_cast<double*>(scr.p), st, gate))
      return EIG_ECUDA;
    const double u = sizeof(T) == 4 ? 5.960464477539063e-08
                                    : (sizeof(T) == 8 && A == Arith::DF64 ? 1.7763568394002505e-15
                                                                         : 1.1102230246251565e-16);
    if (chol_rinv(w, n, static_cast<double*>(G.p), w, static_cast<double*>(Rinv.p), static_cast<double*>(work.p),
                  fl + slot, st, gate, u))
      return EIG_ECUDA;
    if (stage_coef<A>(w, w, static_cast<double*>(Rinv.p), w, static_cast<S*>(Cs.p), w, 1.0, st, gate))
      return EIG_ECUDA;
    if (update<A>(n, src, static_cast<S*>(Cs.p), w, dst, 0.0, st, gate)) return EIG_ECUDA;
    return EIG_OK;
  };
  int rc;
  if ((rc = pass(Wb, Tb, 0, nullptr))) return rc;
  // shifted first pass -> extra pass (shifted CholeskyQR3)
  if ((rc = pass(Tb, Wb, 2, fl + 0))) return rc;
  if (copy_blk<T>(n, Wb, Tb, st, fl + 0)) return EIG_ECUDA;
  if ((rc = pass(Tb, Wb, 1, nullptr))) return rc;
  int hf[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(hf, fl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
    return EIG_ECUDA;
  if (hf[0] == 2 || hf[1] == 2 || hf[2] == 2) return EIG_EBREAKDOWN;
  if (status_out) *status_out = hf[0];
  return EIG_OK;
}

}  // namespace

extern "C" {

int eig_convert(int64_t count, const void* src, int sdt, void* dst, int ddt, void* stream) {
  if (count < 0 || (count > 0 && (!src || !dst))) return EIG_EINVAL;
  if (sdt < EIG_F64 || sdt > EIG_DF64 || ddt < EIG_F64 || ddt > EIG_DF64) return EIG_EINVAL;
  return cuda_status(convert2d(1, count, src, count, sdt, dst, count, ddt, static_cast<cudaStream_t>(stream)));
}

int eig_spmm(int64_t n, const int32_t* rowptr, const int32_t* colind, const void* val, int dtype, int w,
             const void* V, int64_t ldv, void* Y, int64_t ldy, double alpha, double beta, const void* U,
             int64_t ldu, double gamma, void* stream) {
  if (n < 0 || w < 0 || w > 1024 || ldv < w || ldy < w) return EIG_EINVAL;
  if (n > 0 && w > 0 && (!rowptr || !colind || !val || !V || !Y)) return EIG_EINVAL;
  if (gamma != 0.0 && (!U || ldu < w)) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (dtype) {
    case EIG_F64: return spmm_t<Arith::F64>(n, rowptr, colind, val, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
    case EIG_DF64: return spmm_t<Arith::DF64>(n, rowptr, colind, val, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
    case EIG_F32: return spmm_t<Arith::F32>(n, rowptr, colind, val, w, V, ldv, Y, ldy, alpha, beta, U, ldu, gamma, st);
    default: return EIG_EINVAL;
  }
}

int eig_device_status(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) return EIG_ECUDA;
  const int v = tc::tc5_take_error();
  return v < 0 ? EIG_ECUDA : (v ? EIG_ETIMEOUT : EIG_OK);
}

int eig_tc_wait_selftest(int arith, double wait_s, void* stream) {
  if (!arith_tc(arith) || !(wait_s > 0.0) || wait_s > 10.0) return EIG_EINVAL;
  const int ns = arith == EIG_ARITH_DF64_TC ? tc::NS_DF : tc::NS_F64;
  constexpr int64_t n = 1024;
  constexpr int a = 128, b = 64;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t su = (tc_slice_bytes(ns, n, a) + 255) / 256 * 256, sv = tc_slice_bytes(ns, n, b);
  Tmp sl(st), scr(st);
  if (sl.alloc(su + sv) != cudaSuccess) return EIG_ENOMEM;
  if (scr.alloc(sizeof(double) * gram_tc_scratch_elems(ns, n, a, b, false)) != cudaSuccess) return EIG_ENOMEM;
  if (cudaMemsetAsync(sl.p, 0, su + sv, st) != cudaSuccess) return EIG_ECUDA;
  char* pu = static_cast<char*>(sl.p);
  if (tc_wait_selftest(ns, n, a, b, pu, pu + su, static_cast<double*>(scr.p), wait_s, st) != cudaSuccess)
    return EIG_ECUDA;
  return cuda_status(cudaStreamSynchronize(st));
}

int eig_gram(int64_t n, int a, int b, const void* U, int64_t ldu, const void* V, int64_t ldv, int arith, int sym,
             double* G, int64_t ldg, void* stream) {
  if (n < 0 || a < 0 || b < 0 || a > 4096 || b > 4096 || ldu < a || ldv < b || ldg < b) return EIG_EINVAL;
  if ((!arith_ok(arith) && !arith_tc(arith)) || (sym && a != b)) return EIG_EINVAL;
  if (a == 0 || b == 0) return EIG_OK;
  if (!U || !V || !G) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) return cuda_status(cudaMemset2DAsync(G, sizeof(double) * ldg, 0, sizeof(double) * b, a, st));
  switch (arith) {
    case EIG_ARITH_DF64_TC: return gram_tc_t<dd>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_F64_TC: return gram_tc_t<double>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_F64: return gram_t<Arith::F64>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_DF64: return gram_t<Arith::DF64>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    case EIG_ARITH_F32: return gram_t<Arith::F32>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
    default: return gram_t<Arith::C32>(n, a, b, U, ldu, V, ldv, sym, G, ldg, st);
  }
}

int eig_block_update(int64_t n, int s, int c, const void* U, int64_t ldu, const double* C, int64_t ldc, void* Y,
                     int64_t ldy, double beta, int arith, void* stream) {
  if (n < 0 || s < 0 || c < 0 || ldu < s || ldc < c || ldy < c || (!arith_ok(arith) && !arith_tc(arith)))
    return EIG_EINVAL;
  if (n == 0 || c == 0) return EIG_OK;
  if (!Y || (s > 0 && (!U || !C))) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (arith) {
    case EIG_ARITH_DF64_TC: return update_tc_t<dd>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    case EIG_ARITH_F64_TC: return update_tc_t<double>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    case EIG_ARITH_F64: return update_t<Arith::F64>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    case EIG_ARITH_DF64: return update_t<Arith::DF64>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    case EIG_ARITH_F32: return update_t<Arith::F32>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
    default: return update_t<Arith::C32>(n, s, c, U, ldu, C, ldc, Y, ldy, beta, st);
  }
}

int eig_residual(int64_t n, int w, const void* X, int64_t ldx, const void* AX, int64_t ldax, const double* lam,
                 const void* tdiag, void* R, int64_t ldr, double* xnorm2, double* rnorm2, int dtype, void* stream) {
  if (n < 0 || w < 0 || ldx < w || ldax < w || (R && ldr < w)) return EIG_EINVAL;
  if (w == 0) return EIG_OK;
  if (!X || !AX || !lam || !xnorm2 || !rnorm2) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (dtype) {
    case EIG_F64: return residual_t<Arith::F64>(n, w, X, ldx, AX, ldax, lam, tdiag, R, ldr, xnorm2, rnorm2, st);
    case EIG_DF64: return residual_t<Arith::DF64>(n, w, X, ldx, AX, ldax, lam, tdiag, R, ldr, xnorm2, rnorm2, st);
    case EIG_F32: return residual_t<Arith::F32>(n, w, X, ldx, AX, ldax, lam, tdiag, R, ldr, xnorm2, rnorm2, st);
    default: return EIG_EINVAL;
  }
}

int eig_cholqr2(int64_t n, int w, void* W, int64_t ldw, int arith, int* status_out, void* stream) {
  if (n < 0 || w < 0 || w > 1024 || ldw < w || !arith_ok(arith)) return EIG_EINVAL;
  if (w == 0) return EIG_OK;
  if (!W || n < w) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (arith) {
    case EIG_ARITH_F64: return cholqr2_t<Arith::F64>(n, w, W, ldw, status_out, st);
    case EIG_ARITH_DF64: return cholqr2_t<Arith::DF64>(n, w, W, ldw, status_out, st);
    case EIG_ARITH_F32: return cholqr2_t<Arith::F32>(n, w, W, ldw, status_out, st);
    default: return cholqr2_t<Arith::C32>(n, w, W, ldw, status_out, st);
  }
}

int eig_syev(int s, const double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* stream) {
  if (s < 0 || s > 4096 || lda < s || ldz < s) return EIG_EINVAL;
  if (s == 0) return EIG_OK;
  if (!A || !lam || !Z) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Tmp work(st), flag(st);
  if (work.alloc(syev64_work_bytes(s)) || flag.alloc(16)) return EIG_ENOMEM;
  if (cudaMemsetAsync(flag.p, 0, 16, st)) return EIG_ECUDA;
  if (syev64(s, A, lda, lam, Z, ldz, work.p, static_cast<int*>(flag.p), st)) return EIG_ECUDA;
  int hf = 0;
  if (cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
    return EIG_ECUDA;
  return hf ? EIG_EBREAKDOWN : EIG_OK;
}

int eig_hl_trick(int s, int nnow, int nlock, const double* Z, int64_t ldz, double* CP, int64_t ldcp, void* stream) {
  if (s <= 0 || nnow <= 0 || nlock < 0 || nlock >= nnow || nnow > s || ldz < s || ldcp < nnow - nlock)
    return EIG_EINVAL;
  if (s - nnow < nnow - nlock) return EIG_EINVAL;
  if (!Z || !CP) return EIG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Tmp work(st);
  if (work.alloc(hl_work_bytes(s, nnow, nlock))) return EIG_ENOMEM;
  return cuda_status(hl_trick(s, nnow, nlock, Z, ldz, CP, ldcp, work.p, st));
}

}  // extern "C"
