// Host drivers of the block eigensolvers and the C ABI (include/eig_gb300.h).
//
// LOBPCG with soft locking (arXiv:2409.05572, Algorithm 3) and subspace
// iteration with a Chebyshev filter (Algorithm 1), both inside the
// shrink-and-expand framework (Algorithm 5) driven by the fix / slope / slopek
// strategies (Algorithms 6 and 7).  Every n-sized step runs in this library's
// kernels on one stream; the host crosses to the device once per iteration to
// read the residual norms of Eq. conv (a few hundred bytes) and takes the
// strategy decision.
//
// Device layout: S = [X | P | W] and AS = [AX | AP | AW] live in row-major
// n x LDS buffers (LDS = 3 k_max rounded up to 4) with X at column 0, P at
// k_max, W at 2 k_max; two copies of each are used in turn (the block update
// reads S and writes the next X, P).  Active columns are prefixes (plus a
// column offset for P after soft locking), so shrinking and expanding are
// width changes; S_drop is kept in its own n x 2(k_max - nes) buffer.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include "blocks.cuh"
#include "tc.cuh"
#include "small.cuh"

using namespace eig;

// ---------------------------------------------------------------------------
// Shrink-and-expand strategies (Algorithms 6 and 7, Eqs. ckslope/ckslopek,
// warm-up rule).  Readings: the fix clock starts at the first shrink j0
// (expansions when (j - j0 + js) mod je == 0 with nnow == nes, shrinks when
// (j - j0) mod je == 0 with nnow > nes); slope/slopek shrink js iterations
// after each expansion and expand when mu * c < c_max, c_max being the largest
// slope since the last shrink including the current one.
// ---------------------------------------------------------------------------
namespace {

struct SEStrategy {
  int kind = EIG_NONE, nes = 0, nex = 0;
  int je = 12, js = 2, jp = 10, j_warm = 5;
  double mu = 1.1, r_warm = 1e-4;
  bool warm_first = false;  // warm-up gate on the first pair's residual
  std::vector<double> r;    // r[j] for j >= 1 (r[0] unused)
  std::vector<double> r1;   // residual of the first Ritz pair, same indexing
  bool warmed = false;
  int j0 = -1, j_exp = -1;
  bool has_cmax = false;
  double c_max = 0.0;
  int n_shrink = 0, n_expand = 0;

  static double lg(double x) { return std::log10(std::max(x, 1e-300)); }
  void record(int j, double rj, double r1j) {
    if ((int)r.size() <= j) {
      r.resize(j + 1, -1.0);
      r1.resize(j + 1, -1.0);
    }
    r[j] = rj;
    r1[j] = r1j;
  }
  // drop the records from iteration j on
  void forget(int j) {
    r.resize(j);
    r1.resize(j);
  }
  bool have(int j) const { return j >= 1 && j < (int)r.size() && r[j] >= 0.0; }
  bool slope(int j, double* c) const {
    if (kind == EIG_SLOPE) {
      if (!have(j - 1)) return false;
      *c = lg(r[j - 1]) - lg(r[j]);
      return true;
    }
    if (kind == EIG_SLOPEK) {
      if (j < jp || !have(j - jp)) return false;
      *c = (lg(r[j - jp]) - lg(r[j])) / jp;
      return true;
    }
    return false;
  }
  bool ifexpand(int j, int nnow) {
    if (kind == EIG_NONE || !warmed) return false;
    bool go = false;
    if (kind == EIG_FIX) {
      go = nnow == nes && ((j - j0 + js) % je) == 0;
    } else {
      double c;
      if (nnow == nes && slope(j, &c)) {
        c_max = has_cmax ? std::max(c_max, c) : c;
        has_cmax = true;
        go = mu * c < c_max;
      }
    }
    if (go) {
      j_exp = j;
      ++n_expand;
    }
    return go;
  }
  bool ifshrink(int j, int nnow) {
    if (kind == EIG_NONE || nnow <= nes) return false;
    bool go;
    if (!warmed) {
      go = j >= j_warm && have(j) && (warm_first ? r1[j] : r[j]) <= r_warm;
      if (go) {
        warmed = true;
        j0 = j;
      }
    } else if (kind == EIG_FIX) {
      go = ((j - j0) % je) == 0;
    } else {
      go = j_exp >= 0 && (j - j_exp) == js;
    }
    if (go) {
      has_cmax = false;
      ++n_shrink;
    }
    return go;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
// SpMM rows longer than this are split over the warps of a CTA
constexpr int HEAVY_MIN = 512;

// max_i sum_j |a_ij| of host CSR arrays (an upper bound of ||A||_2 for a
// symmetric A, and of the spectrum's magnitude)
double gershgorin_bound(int64_t n, const int32_t* rp, const void* val, int val_dtype) {
  double best = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      r += val_dtype == EIG_F32 ? std::fabs(double(static_cast<const float*>(val)[k]))
                                : std::fabs(static_cast<const double*>(val)[k]);
    best = std::max(best, r);
  }
  return best;
}

struct eig_handle {
  int64_t n = 0, nnz = 0;
  int nev = 0, kmax = 0, nes = 0, strategy = 0;
  eig_options opt{};
  cudaStream_t st = nullptr;
  int LDS = 0, hdrop = 0, wtw = 0, cqmax = 0;

  // CSR (device)
  int32_t *rowptr = nullptr, *colind = nullptr;
  double* val64 = nullptr;
  dd* valdd = nullptr;
  float* val32 = nullptr;
  bool own_idx = false;
  int32_t* heavy = nullptr;  // rows with more than HEAVY_MIN nonzeros (device)
  int nheavy = 0;
  // Jacobi diagonal and null vector, per storage format
  double* t64 = nullptr;
  dd* tdd = nullptr;
  float* t32 = nullptr;
  double* u64 = nullptr;
  dd* udd = nullptr;
  float* u32 = nullptr;
  // n-sized blocks (bytes for 8-byte elements)
  void* S[2] = {nullptr, nullptr};
  void* AS[2] = {nullptr, nullptr};
  void* Wt = nullptr;
  void* Sd = nullptr;
  // bf16 slices of the two Gram operands (opt.gram_tc, double-float blocks)
  void* tcU = nullptr;
  void* tcV = nullptr;
  void* tcC = nullptr;  // slices of the update coefficients
  // slices of the projection basis Q of an orthogonalisation, both layouts
  // (kept for the two projections of one orth())
  void* tcQc = nullptr;
  void* tcQr = nullptr;
  int qcmax = 0;
  int tcns = 0;  // slices per value (6 double-float, 7 float64)
  int64_t tcrows = 0;     // rows held by tcU / tcV (n, or the chunk of tc_chunk_rows)
  double* Gt = nullptr;   // Gram of one row chunk (chunked tensor-core products)
  // small float64 work
  int smax = 0;
  double *Gp = nullptr, *Rinv = nullptr, *cholw = nullptr, *Z = nullptr, *lamd = nullptr, *CP = nullptr;
  double *gscr = nullptr, *rscr = nullptr, *xn = nullptr, *rn = nullptr;
  void* Cs = nullptr;
  void* syevw = nullptr;
  void* hlw = nullptr;
  int* flags = nullptr;  // device: [0..3] CholQR statuses, [4] syev status
  double* hpin = nullptr;
  // results
  double* V = nullptr;
  std::vector<double> lam, resid, history;
  std::vector<int> widths;
  int status = EIG_OK, iters = 0, n_shrink = 0, n_expand = 0;
  double time_ms = 0.0;
  int64_t launches = 0;
  cudaError_t cuda_err = cudaSuccess;
  // per-kernel-class statistics (opt.profile)
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    double flops, bytes;
  };
  std::vector<Rec> pend;
  std::vector<cudaEvent_t> evpool;
  double kst[EIG_NKCLASS][4] = {};
};

#define CK(x)                      \
  do {                             \
    cudaError_t e_ = (x);          \
    if (e_ != cudaSuccess) {       \
      h->cuda_err = e_;            \
      return EIG_ECUDA;            \
    }                              \
  } while (0)

namespace {

constexpr int F_CHOL1 = 0, F_CHOL2 = 1, F_CHOL3 = 2, F_SYEV = 4, NFLAGS = 8;

// Diagnostics of a debug build (compiled with -DEIG_DEBUG_LEVEL=1 or 2;
// the shipped library has level 0 and no diagnostic path): 1 prints the
// block norms of every step and the residual test of every iteration, 2 also
// re-solves every projected eigenproblem with the float64 QL path and prints
// the largest eigenvalue difference.
#ifndef EIG_DEBUG_LEVEL
#define EIG_DEBUG_LEVEL 0
#endif
constexpr int debug_level() { return EIG_DEBUG_LEVEL; }
constexpr bool debug_on() { return EIG_DEBUG_LEVEL >= 1; }

// CUDA-event bracket of one kernel class when profiling is on
cudaEvent_t ev_get(eig_handle* h) {
  if (!h->evpool.empty()) {
    cudaEvent_t e = h->evpool.back();
    h->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
struct Prof {
  eig_handle* h;
  int cls;
  double fl, by;
  cudaEvent_t a = nullptr;
  Prof(eig_handle* hh, int c, double flops, double bytes) : h(hh), cls(c), fl(flops), by(bytes) {
    if (h->opt.profile) {
      a = ev_get(h);
      cudaEventRecord(a, h->st);
    }
  }
  ~Prof() {
    if (a) {
      cudaEvent_t b = ev_get(h);
      cudaEventRecord(b, h->st);
      h->pend.push_back({a, b, cls, fl, by});
    }
  }
};
// resolve recorded brackets (stream already synchronised)
void prof_flush(eig_handle* h) {
  for (auto& r : h->pend) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    h->kst[r.cls][0] += 1.0;
    h->kst[r.cls][1] += ms;
    h->kst[r.cls][2] += r.flops;
    h->kst[r.cls][3] += r.bytes;
    h->evpool.push_back(r.a);
    h->evpool.push_back(r.b);
  }
  h->pend.clear();
}

template <typename T>
Blk<T> view(void* base, int64_t ld, int col, int w) {
  Blk<T> b;
  b.add(static_cast<T*>(base) + col, ld, w);
  return b;
}
template <typename T>
Blk<T> cat(const Blk<T>& a, const Blk<T>& b) {
  Blk<T> r = a;
  for (int t = 0; t < b.nseg; ++t) r.add(b.ptr[t], b.ld[t], b.start[t + 1] - b.start[t]);
  return r;
}

template <typename T>
bool same_blk(const Blk<T>& a, const Blk<T>& b) {
  if (a.nseg != b.nseg || a.width != b.width) return false;
  for (int t = 0; t < a.nseg; ++t)
    if (a.ptr[t] != b.ptr[t] || a.ld[t] != b.ld[t] || a.start[t + 1] != b.start[t + 1]) return false;
  return true;
}

// the Gram products and updates of the float64 and double-float blocks run
// on the tensor cores (slice buffers); slices per value of the form's blocks
bool uses_gram_tc(const eig_options& o) { return o.gram_tc != 0; }
int tc_slices(int form) { return form == EIG_FORM_F64 ? tc::NS_F64 : tc::NS_DF; }
// rows held by the slice buffers: all n, or the chunk of tc_chunk_rows
int64_t tc_rows_of(int64_t n, int chunk) { return (chunk > 0 && chunk < n) ? int64_t(chunk) : n; }

// the view of rows r0 .. of a block
template <typename T>
Blk<T> rows_from(const Blk<T>& b, int64_t r0) {
  Blk<T> r = b;
  for (int t = 0; t < b.nseg; ++t) r.ptr[t] = b.ptr[t] + r0 * b.ld[t];
  return r;
}

// one slice buffer: a Gram operand (K = n, up to w columns) or an update's
// left operand (K = up to w columns, n rows)
size_t tc_operand_bytes(int ns, int64_t n, int w) {
  return std::max(tc_slice_bytes(ns, n, w), tc_slice_bytes(ns, w, n));
}

template <Arith A> struct FormData;
template <> struct FormData<Arith::DF64> {
  static const dd* val(eig_handle* h) { return h->valdd; }
  static const dd* tdiag(eig_handle* h) { return h->tdd; }
  static dd* u0(eig_handle* h) { return h->udd; }
};
template <> struct FormData<Arith::F64> {
  static const double* val(eig_handle* h) { return h->val64; }
  static const double* tdiag(eig_handle* h) { return h->t64; }
  static double* u0(eig_handle* h) { return h->u64; }
};
template <> struct FormData<Arith::F32> {
  static const float* val(eig_handle* h) { return h->val32; }
  static const float* tdiag(eig_handle* h) { return h->t32; }
  static float* u0(eig_handle* h) { return h->u32; }
};

// AU: arithmetic of SpMM / update / residual; AG: arithmetic of the Gram
// products (same storage type).
template <Arith AU, Arith AG>
struct Ops {
  using T = typename Pol<AU>::T;
  using SU = typename Pol<AU>::S;
  eig_handle* h;
  explicit Ops(eig_handle* hh) : h(hh) {}
  cudaStream_t st() const { return h->st; }
  Csr<AU> csr() const {
    Csr<AU> c;
    c.n = h->n;
    c.rowptr = h->rowptr;
    c.colind = h->colind;
    c.val = FormData<AU>::val(h);
    c.heavy = h->heavy;
    c.nheavy = h->nheavy;
    c.heavy_min = HEAVY_MIN;
    return c;
  }
  int64_t ld() const { return h->LDS; }

  static constexpr double E = sizeof(T);
  // unit roundoff of the block storage (shift of the shifted CholeskyQR)
  static constexpr double kUnitRound = sizeof(T) == 4 ? 5.960464477539063e-08
                                       : (std::is_same<T, dd>::value ? 1.7763568394002505e-15
                                                                     : 1.1102230246251565e-16);
  // Q of the current orth() whose slices (both layouts) are in tcQc / tcQr
  bool qcache = false;
  Blk<T> qblk;
  bool q_cached(const Blk<T>& U) const { return qcache && same_blk(U, qblk); }

  // G = U^T V into h->Gp (leading dimension b)
  int gram(const Blk<T>& U, const Blk<T>& V, bool sym, const int* gate = nullptr) {
    const double nn = double(h->n), a = U.width, b = V.width;
    const bool same = U.ptr[0] == V.ptr[0];
    Prof p(h, EIG_K_GRAM, sym ? nn * a * (b + 1) : 2.0 * nn * a * b, E * nn * (same ? a : a + b));
    if constexpr (AG == Arith::DF64 || AG == Arith::F64) {
      if (h->tcU) {  // tensor-core product on exact bf16 slices
        const bool one = same_blk(U, V);
        if (h->tcrows < h->n) {
          // row chunks: G = sum over chunks of U_c^T V_c, added in chunk order
          for (int64_t r0 = 0; r0 < h->n; r0 += h->tcrows) {
            const int64_t rr = std::min(h->tcrows, h->n - r0);
            const Blk<T> Uc = rows_from(U, r0);
            CK(tc_slice_cols(rr, Uc, h->tcU, st(), gate));
            if (!one) CK(tc_slice_cols(rr, rows_from(V, r0), h->tcV, st(), gate));
            double* dst = r0 == 0 ? h->Gp : h->Gt;
            CK(gram_tc_product(h->tcns, rr, U.width, V.width, h->tcU, one ? h->tcU : h->tcV, sym, dst, V.width,
                               h->gscr, st(), gate));
            if (r0 > 0)
              CK(eig::axpby<Arith::F64>(U.width, V.width, h->Gp, V.width, 1.0, h->Gt, V.width, 1.0, h->Gp,
                                        V.width, st()));
          }
          return EIG_OK;
        }
        const bool ucached = q_cached(U);
        void* su = ucached ? h->tcQc : h->tcU;
        if (!ucached) CK(tc_slice_cols(h->n, U, h->tcU, st(), gate));
        if (!one) CK(tc_slice_cols(h->n, V, h->tcV, st(), gate));
        CK(gram_tc_product(h->tcns, h->n, U.width, V.width, su, one ? su : h->tcV, sym, h->Gp, V.width, h->gscr,
                           st(), gate));
        return EIG_OK;
      }
    }
    CK(eig::gram<AG>(h->n, U, V, sym, h->Gp, V.width, h->gscr, st(), gate));
    return EIG_OK;
  }
  // Y = U (scale * C) + beta Y with C float64 (s x c, ldc)
  int upd(const Blk<T>& U, const double* C, int64_t ldc, int c, double scale, const Blk<T>& Y, double beta,
          const int* gate = nullptr) {
    if constexpr (AU == Arith::DF64 || AU == Arith::F64) {
      if (h->tcU && U.width > 0 && c > 0) {  // tensor-core product on exact bf16 slices
        {
          Prof p(h, EIG_K_OTHER, 0.0, 0.0);
          CK(tc_slice_coef(h->tcns, U.width, c, C, ldc, scale, h->tcC, st(), gate));
        }
        const double nn = double(h->n);
        Prof p(h, EIG_K_UPDATE, 2.0 * nn * U.width * c, E * nn * (U.width + c * (beta != 0.0 ? 2.0 : 1.0)));
        if (h->tcrows < h->n) {  // row chunks: each output row needs only its own U row
          for (int64_t r0 = 0; r0 < h->n; r0 += h->tcrows) {
            const int64_t rr = std::min(h->tcrows, h->n - r0);
            CK(tc_slice_rows(rr, rows_from(U, r0), h->tcU, st(), gate));
            CK(update_tc_product(rr, U.width, c, h->tcU, h->tcC, rows_from(Y, r0), beta, st(), gate));
          }
          return EIG_OK;
        }
        const bool ucached = q_cached(U);
        if (!ucached) CK(tc_slice_rows(h->n, U, h->tcU, st(), gate));
        CK(update_tc_product(h->n, U.width, c, ucached ? h->tcQr : h->tcU, h->tcC, Y, beta, st(), gate));
        return EIG_OK;
      }
    }
    {
      Prof p(h, EIG_K_OTHER, 0.0, 0.0);
      CK(stage_coef<AU>(U.width, c, C, ldc, static_cast<SU*>(h->Cs), c, scale, st(), gate));
    }
    const double nn = double(h->n);
    Prof p(h, EIG_K_UPDATE, 2.0 * nn * U.width * c, E * nn * (U.width + c * (beta != 0.0 ? 2.0 : 1.0)));
    CK(eig::update<AU>(h->n, U, static_cast<SU*>(h->Cs), c, Y, beta, st(), gate));
    return EIG_OK;
  }
  // one CholeskyQR pass: dst = src R^{-1}; status into flags[slot]
  int cholqr(const Blk<T>& src, const Blk<T>& dst, int slot, const int* gate = nullptr) {
    const int w = src.width;
    if (w > h->cqmax) return EIG_EINVAL;  // work buffers are sized for cqmax
    int rc = gram(src, src, true, gate);
    if (rc) return rc;
    {
      Prof p(h, EIG_K_CHOL, 2.0 * w * double(w) * w / 3.0, 0.0);
      CK(chol_rinv(w, h->n, h->Gp, w, h->Rinv, h->cholw, h->flags + slot, st(), gate, kUnitRound));
    }
    return upd(src, h->Rinv, w, w, 1.0, dst, 0.0, gate);
  }
  double spmm_bytes(int w, int terms) const {
    return (4.0 + E) * double(h->nnz) + 4.0 * double(h->n + 1) + E * double(h->n) * w * (1 + terms);
  }
  // debug (EIG_DEBUG=2): eigenvalues of the same projected matrix by the
  // float64 QL path, compared with the refined eigensolver's
  void compare_syev(int s) {
    std::vector<double> ap(size_t(s) * s), l1(s), l2(s);
    cudaMemcpyAsync(ap.data(), h->Gp, sizeof(double) * ap.size(), cudaMemcpyDeviceToHost, st());
    cudaMemcpyAsync(l1.data(), h->lamd, sizeof(double) * s, cudaMemcpyDeviceToHost, st());
    double *dA = nullptr, *dl = nullptr, *dZ = nullptr;
    void* wk = nullptr;
    int* fl = nullptr;
    cudaMalloc(&dA, sizeof(double) * ap.size());
    cudaMalloc(&dl, sizeof(double) * s);
    cudaMalloc(&dZ, sizeof(double) * ap.size());
    cudaMalloc(&wk, syev_qr64_work_bytes(s));
    cudaMalloc(&fl, 16);
    cudaMemcpyAsync(dA, h->Gp, sizeof(double) * ap.size(), cudaMemcpyDeviceToDevice, st());
    syev_qr64(s, dA, s, dl, dZ, s, wk, fl, st());
    cudaMemcpyAsync(l2.data(), dl, sizeof(double) * s, cudaMemcpyDeviceToHost, st());
    cudaStreamSynchronize(st());
    double nrm = 0.0, worst = 0.0;
    int wi = 0;
    for (int i = 0; i < s; ++i) nrm = std::max(nrm, std::fabs(l2[i]));
    for (int i = 0; i < s; ++i)
      if (std::fabs(l1[i] - l2[i]) > worst) {
        worst = std::fabs(l1[i] - l2[i]);
        wi = i;
      }
    std::fprintf(stderr, "[eig]   syev check s=%d: max |dlam|/|A_p| = %.2e at %d (lam %.12f vs %.12f)\n", s,
                 worst / nrm, wi, l1[wi], l2[wi]);
    bool finite = true;
    for (int i = 0; i < s; ++i) finite = finite && std::isfinite(l1[i]);
    cudaFree(dA);
    cudaFree(dl);
    cudaFree(dZ);
    cudaFree(wk);
    cudaFree(fl);
  }
  // debug: min / max column norm of a block (EIG_DEBUG=1 only)
  void dbg(const char* label, const Blk<T>& B) {
    if (!debug_on() || B.width == 0) return;
    if (gram(B, B, true)) return;
    std::vector<double> g(size_t(B.width) * B.width);
    cudaMemcpyAsync(g.data(), h->Gp, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, st());
    cudaStreamSynchronize(st());
    double mn = 1e300, mx = -1e300, off = 0.0;
    int nan = 0, first_nan_col = -1;
    for (int i = 0; i < B.width; ++i) {
      mn = std::min(mn, g[size_t(i) * B.width + i]);
      mx = std::max(mx, g[size_t(i) * B.width + i]);
      for (int j = 0; j < B.width; ++j) {
        const double v = g[size_t(i) * B.width + j];
        if (!std::isfinite(v)) {
          ++nan;
          if (first_nan_col < 0) first_nan_col = j;
        }
        if (i != j) off = std::max(off, std::fabs(v));
      }
    }
    std::fprintf(stderr, "[eig]   %s: w=%d diag(G) in [%.3e, %.3e], max offdiag %.3e, nonfinite %d (col %d)\n",
                 label, B.width, mn, mx, off, nan, first_nan_col);
  }
  // project D against Q (D -= Q Q^T D)
  int project(const Blk<T>& Q, const Blk<T>& D) {
    if (Q.width == 0) return EIG_OK;
    int rc = gram(Q, D, false);
    if (rc) return rc;
    return upd(Q, h->Gp, D.width, D.width, -1.0, D, 1.0);
  }
  // Orthonormal basis of (I - Q Q^T) Dsrc, written to Ddst: two passes of
  // projection + CholeskyQR (a third CholeskyQR when the first needed the
  // shift).  Dmid is scratch; Dsrc is clobbered (Ddst may alias Dsrc).
  int orth(const Blk<T>& Q, const Blk<T>& Dsrc, const Blk<T>& Dmid, const Blk<T>& Ddst, bool trace = false) {
    // tensor-core form: Q does not change during the orthogonalisation, so
    // its slices are made once, in both layouts, for both projections
    struct Clear {
      bool& f;
      ~Clear() { f = false; }
    } clear{qcache};
    if constexpr (AU == AG && (AU == Arith::DF64 || AU == Arith::F64)) {
      if (h->tcQc && Q.width > 0 && Q.width <= h->qcmax) {
        const double nn = double(h->n);
        {
          Prof p(h, EIG_K_GRAM, 0.0, E * nn * Q.width);
          CK(tc_slice_cols(h->n, Q, h->tcQc, st()));
        }
        {
          Prof p(h, EIG_K_UPDATE, 0.0, E * nn * Q.width);
          CK(tc_slice_rows(h->n, Q, h->tcQr, st()));
        }
        qcache = true;
        qblk = Q;
      }
    }
    int rc;
    if ((rc = project(Q, Dsrc))) return rc;
    if (trace) dbg("  after projection 1", Dsrc);
    if ((rc = cholqr(Dsrc, Dmid, F_CHOL1))) return rc;
    if (trace) {
      int f[4];
      const int w = Dsrc.width;
      std::vector<double> g(size_t(w) * w), ri(size_t(w) * w);
      cudaMemcpyAsync(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, st());
      cudaMemcpyAsync(g.data(), h->Gp, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, st());
      cudaMemcpyAsync(ri.data(), h->Rinv, sizeof(double) * ri.size(), cudaMemcpyDeviceToHost, st());
      cudaStreamSynchronize(st());
      std::fprintf(stderr, "[eig]   flags after cholqr 1: %d %d %d\n", f[0], f[1], f[2]);
      for (int i = 0; i < std::min(w, 4); ++i) {
        std::fprintf(stderr, "[eig]   G[%d] =", i);
        for (int j = 0; j < std::min(w, 6); ++j) std::fprintf(stderr, " %.4e", g[size_t(i) * w + j]);
        std::fprintf(stderr, " | Rinv:");
        for (int j = 0; j < std::min(w, 6); ++j) std::fprintf(stderr, " %.4e", ri[size_t(i) * w + j]);
        std::fprintf(stderr, "\n");
      }
      dbg("  after cholqr 1", Dmid);
    }
    // conditional third pass (shifted CholeskyQR3): Dmid -> Dsrc -> Dmid
    if ((rc = cholqr(Dmid, Dsrc, F_CHOL3, h->flags + F_CHOL1))) return rc;
    {
      Prof p(h, EIG_K_OTHER, 0.0, 0.0);
      CK(copy_blk<T>(h->n, Dsrc, Dmid, st(), h->flags + F_CHOL1));
    }
    if ((rc = project(Q, Dmid))) return rc;
    return cholqr(Dmid, Ddst, F_CHOL2);
  }
  int spmm(const T* V, int64_t ldv, int w, T* Y, int64_t ldy) {
    Prof p(h, EIG_K_SPMM, 2.0 * double(h->nnz) * w, spmm_bytes(w, 1));
    CK(eig::spmm<AU>(csr(), w, V, ldv, Y, ldy, 1.0, 0.0, nullptr, 0, 0.0, st()));
    return EIG_OK;
  }
  int spmm3(const T* V, int w, T* Y, double alpha, double beta, const T* U, double gamma) {
    Prof p(h, EIG_K_SPMM, 2.0 * double(h->nnz) * w + 4.0 * double(h->n) * w, spmm_bytes(w, 3));
    CK(eig::spmm<AU>(csr(), w, V, ld(), Y, ld(), alpha, beta, U, ld(), gamma, st()));
    return EIG_OK;
  }
  int spmm_blk(const Blk<T>& V, const Blk<T>& Y) {
    for (int t = 0; t < V.nseg; ++t) {
      const int w = V.start[t + 1] - V.start[t];
      // Y has the same segmentation by construction
      Prof p(h, EIG_K_SPMM, 2.0 * double(h->nnz) * w, spmm_bytes(w, 1));
      CK(eig::spmm<AU>(csr(), w, V.ptr[t], V.ld[t], Y.ptr[t], Y.ld[t], 1.0, 0.0, nullptr, 0, 0.0, st()));
    }
    return EIG_OK;
  }
  // Rayleigh-Ritz: Gp = S^T AS, then Z, lamd
  int rr(const Blk<T>& S, const Blk<T>& ASb) {
    int rc = gram(S, ASb, true);
    if (rc) return rc;
    const double sw = S.width;
    Prof p(h, EIG_K_SYEV, (4.0 / 3.0 + 6.0) * sw * sw * sw, 0.0);
    // float64 form: the float64 eigensolver; double-float and mixed forms:
    // the float32 decomposition refined in double-float
    if constexpr (AU == Arith::F64)
      CK(syev64(S.width, h->Gp, S.width, h->lamd, h->Z, S.width, h->syevw, h->flags + F_SYEV, st()));
    else
      CK(syev(S.width, h->Gp, S.width, h->lamd, h->Z, S.width, h->syevw, h->flags + F_SYEV, st()));
    if constexpr (debug_level() >= 2) compare_syev(S.width);
    return EIG_OK;
  }
  int hl(int s, int nnow, int nlock, int npn) {
    Prof p(h, EIG_K_HL, 4.0 * double(s) * (s - nnow) * (nnow - nlock), 0.0);
    CK(hl_trick(s, nnow, nlock, h->Z, s, h->CP, npn, h->hlw, h->st));
    return EIG_OK;
  }
  int axpby_(int w, const T* U, double a, const T* V, double b, T* Y) {
    Prof p(h, EIG_K_OTHER, 4.0 * double(h->n) * w, 3.0 * E * double(h->n) * w);
    CK(eig::axpby<AU>(h->n, w, U, ld(), a, V, ld(), b, Y, ld(), st()));
    return EIG_OK;
  }
  // residual norms (and R into Rdst when non-null); copies norms, lam and
  // flags to the host and synchronises.
  // residual + asynchronous copy of norms, Ritz values and status flags to
  // the host (pinned); the caller synchronises the stream before reading.
  int resid_launch(const T* X, const T* AX, int w, T* Rdst, bool precond) {
    const T* td = precond ? FormData<AU>::tdiag(h) : nullptr;
    {
      Prof p(h, EIG_K_RESIDUAL, 6.0 * double(h->n) * w, E * double(h->n) * w * (Rdst ? 3.0 : 2.0));
      CK(eig::residual<AU>(h->n, w, X, ld(), AX, ld(), h->lamd, td, Rdst, ld(), h->xn, h->rn, h->rscr, st()));
    }
    CK(cudaMemcpyAsync(h->hpin, h->xn, sizeof(double) * w, cudaMemcpyDeviceToHost, st()));
    CK(cudaMemcpyAsync(h->hpin + h->kmax, h->rn, sizeof(double) * w, cudaMemcpyDeviceToHost, st()));
    CK(cudaMemcpyAsync(h->hpin + 2 * h->kmax, h->lamd, sizeof(double) * w, cudaMemcpyDeviceToHost, st()));
    CK(cudaMemcpyAsync(h->hpin + 3 * h->kmax, h->flags, sizeof(int) * NFLAGS, cudaMemcpyDeviceToHost, st()));
    CK(cudaMemsetAsync(h->flags, 0, sizeof(int) * NFLAGS, st()));
    return EIG_OK;
  }
};

// Eq. conv / Eq. rk from the host copies of the norms
struct ConvInfo {
  double r = 0.0;   // r^(j) of Eq. rk (largest over the first nev pairs)
  double r1 = 0.0;  // Eq. conv of the first Ritz pair
  int nlock = 0;
  bool breakdown = false;
};

ConvInfo conv_test(eig_handle* h, int w) {
  ConvInfo ci;
  const double* xn = h->hpin;
  const double* rn = h->hpin + h->kmax;
  const double* lam = h->hpin + 2 * h->kmax;
  const int* fl = reinterpret_cast<const int*>(h->hpin + 3 * h->kmax);
  const double nA = h->opt.normA;
  double r = 0.0;
  bool prefix = true;
  for (int i = 0; i < h->nev && i < w; ++i) {
    const double x = std::sqrt(std::max(xn[i], 0.0));
    const double rho = std::sqrt(std::max(rn[i], 0.0)) / (nA * x + x * std::fabs(lam[i]));
    const double rr = std::isfinite(rho) ? rho : 1e300;
    if (i == 0) ci.r1 = rr;
    r = std::max(r, rr);
    if (prefix && rr <= h->opt.tol)
      ++ci.nlock;
    else
      prefix = false;
  }
  ci.r = r;
  ci.breakdown = fl[F_CHOL1] == 2 || fl[F_CHOL2] == 2 || fl[F_CHOL3] == 2 || fl[F_SYEV] != 0;
  if (debug_on())
    std::fprintf(stderr, "[eig] j=%d w=%d r=%.3e nlock=%d flags chol=%d/%d/%d syev=%d\n", h->iters + 1, w, r,
                 ci.nlock, fl[F_CHOL1], fl[F_CHOL2], fl[F_CHOL3], fl[F_SYEV]);
  return ci;
}

int finish(eig_handle* h, int status);

// ---------------------------------------------------------------------------
// LOBPCG with soft locking and shrink-and-expand (Algorithm 3).
// Phase state carried between precision phases of the mixed form.
// ---------------------------------------------------------------------------
struct LState {
  int cur = 0;       // which S / AS buffer holds the iterate
  int nnow = 0;      // active width of X
  int np = 0;        // width of P
  int poff = 0;      // column offset of P inside its slot
  int nlock = 0;
  bool have_drop = false;
  int n_exp = 0;     // expansions so far (block index of the 'Random' draws)
  int j = 0;         // last iteration done
  SEStrategy se;
};

// element format code of a block type
template <typename T> constexpr int fmt_of() {
  return sizeof(T) == 4 ? EIG_F32 : (std::is_same<T, dd>::value ? EIG_DF64 : EIG_F64);
}

template <Arith AU, Arith AG>
int lobpcg_init(eig_handle* h, LState& L) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  const int64_t ld = h->LDS;
  const int k = h->kmax;
  // X0 (host or device float64) -> device staging in S[1] -> X slot of S[0]
  // in the element format of the phase
  CK(cudaMemcpyAsync(h->S[1], h->opt.X0, sizeof(double) * size_t(h->n) * k, cudaMemcpyDefault, h->st));
  const int fmt = sizeof(T) == 4 ? EIG_F32 : (std::is_same<T, dd>::value ? EIG_DF64 : EIG_F64);
  CK(convert2d(h->n, k, h->S[1], k, EIG_F64, h->S[0], ld, fmt, h->st));
  Blk<T> X = view<T>(h->S[0], ld, 0, k);
  Blk<T> Q;
  if (h->opt.deflate_ones) Q.add(FormData<AU>::u0(h), 1, 1);
  Blk<T> mid = view<T>(h->Wt, h->wtw, 0, k);
  Blk<T> Xd = view<T>(h->S[1], ld, 0, k);
  int rc = o.orth(Q, X, mid, Xd);  // orthonormal X0 in S[1]
  if (rc) return rc;
  Blk<T> AX = view<T>(h->AS[1], ld, 0, k);
  if ((rc = o.spmm_blk(Xd, AX))) return rc;
  if ((rc = o.rr(Xd, AX))) return rc;
  // X <- X Z into buffer 0, AX = A X
  if ((rc = o.upd(Xd, h->Z, k, k, 1.0, view<T>(h->S[0], ld, 0, k), 0.0))) return rc;
  if ((rc = o.spmm(static_cast<T*>(h->S[0]), ld, k, static_cast<T*>(h->AS[0]), ld))) return rc;
  L.cur = 0;
  L.nnow = k;
  L.np = 0;
  L.poff = 0;
  L.nlock = 0;
  L.have_drop = false;
  L.j = 0;
  return EIG_OK;
}

// One LOBPCG iteration is split at its single host crossing: lob_pre
// launches R = T (AX - X Lambda) into the W slot and the copy of the norms to
// the host; after the stream is synchronised lob_post takes the convergence
// and strategy decisions and launches the rest of the iteration.  *done is
// set on convergence, *switched when the residual reached switch_r (the
// iteration is then redone in the next precision).
template <Arith AU, Arith AG>
int lob_pre(eig_handle* h, LState& L) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  T* X = static_cast<T*>(h->S[L.cur]);
  T* AX = static_cast<T*>(h->AS[L.cur]);
  return o.resid_launch(X, AX, L.nnow, X + 2 * h->kmax, h->opt.precond != 0);
}

template <Arith AU, Arith AG>
int lob_post(eig_handle* h, LState& L, double switch_r, bool* done, bool* switched) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  const int64_t ld = h->LDS;
  const int k = h->kmax, nes = h->nes;
  *done = false;
  *switched = false;
  int rc;
  {
    const int j = L.j + 1;
    void* Sc = h->S[L.cur];
    void* ASc = h->AS[L.cur];
    T* X = static_cast<T*>(Sc);
    T* Wslot = X + 2 * k;
    ConvInfo ci = conv_test(h, L.nnow);
    if (ci.breakdown) return EIG_EBREAKDOWN;
    h->history.push_back(ci.r);
    L.se.record(j, ci.r, ci.r1);
    L.j = j;
    h->iters = j;
    if (ci.r <= h->opt.tol) {
      *done = true;
      return EIG_OK;
    }
    if (switch_r > 0.0 && ci.r <= switch_r) {
      // hand over before doing this iteration's update in the next form
      L.j = j - 1;
      h->history.pop_back();
      L.se.forget(j);
      *switched = true;
      return EIG_OK;
    }
    // soft locking: drop the P columns of newly locked X columns
    if (ci.nlock > L.nlock) {
      const int d = std::min(ci.nlock - L.nlock, L.np);
      L.poff += d;
      L.np -= d;
    }
    L.nlock = ci.nlock;
    const int nw = L.nnow - L.nlock;
    Blk<T> Xb = view<T>(Sc, ld, 0, L.nnow);
    Blk<T> Pb = view<T>(Sc, ld, k + L.poff, L.np);
    Blk<T> Q;
    if (h->opt.deflate_ones) Q.add(FormData<AU>::u0(h), 1, 1);
    Q = cat(cat(Q, Xb), Pb);
    Blk<T> Wb = view<T>(Sc, ld, 2 * k + L.nlock, nw);
    Blk<T> Wmid = view<T>(h->Wt, h->wtw, 0, nw);
    if ((rc = o.orth(Q, Wb, Wmid, Wb))) return rc;
    // expansion: re-orthogonalise S_drop against S, append halves to X and P
    if (L.se.ifexpand(j, L.nnow)) {
      if (!L.have_drop) return EIG_EINVAL;
      const int hd = h->hdrop;
      // 'Random' variant (Sec. 6.4): fresh Gaussian columns replace S_drop
      if (h->opt.expand_random)
        CK(gauss_fill(h->n, 2 * hd, h->Sd, 2 * hd, fmt_of<T>(), h->opt.seed, L.n_exp, h->st));
      ++L.n_exp;
      // P must be contiguous from the slot start for the append: move it if offset
      Blk<T> Dsrc = view<T>(h->Sd, 2 * hd, 0, 2 * hd);
      Blk<T> Dmid = view<T>(h->Wt, h->wtw, 0, 2 * hd);
      Blk<T> Ddst = cat(view<T>(Sc, ld, L.nnow, hd), view<T>(Sc, ld, k + L.poff + L.np, hd));
      Blk<T> Sfull = cat(Q, Wb);
      o.dbg("S before expansion", Sfull);
      o.dbg("S_drop before orth", Dsrc);
      if ((rc = o.orth(Sfull, Dsrc, Dmid, Ddst, debug_on()))) return rc;
      o.dbg("S_drop after orth", Ddst);
      Blk<T> ADdst = cat(view<T>(ASc, ld, L.nnow, hd), view<T>(ASc, ld, k + L.poff + L.np, hd));
      if ((rc = o.spmm_blk(Ddst, ADdst))) return rc;
      L.nnow += hd;
      L.np += hd;
      L.have_drop = false;
    }
    Xb = view<T>(Sc, ld, 0, L.nnow);
    Pb = view<T>(Sc, ld, k + L.poff, L.np);
    // AW = A W
    if ((rc = o.spmm(Wslot + L.nlock, ld, nw, static_cast<T*>(ASc) + 2 * k + L.nlock, ld))) return rc;
    Blk<T> Sb = cat(cat(Xb, Pb), Wb);
    Blk<T> ASb = cat(cat(view<T>(ASc, ld, 0, L.nnow), view<T>(ASc, ld, k + L.poff, L.np)),
                     view<T>(ASc, ld, 2 * k + L.nlock, nw));
    const int s = Sb.width;
    h->widths.push_back(L.nnow);
    if ((rc = o.rr(Sb, ASb))) return rc;
    // improved Hetmaniuk-Lehoucq: C = [Z(:, :nnow) | C_P]
    const int npn = L.nnow - L.nlock;
    if ((rc = o.hl(s, L.nnow, L.nlock, npn))) return rc;
    // X, AX <- S C_X, AS C_X ; P, AP <- S C_P, AS C_P (next buffers)
    const int nx = 1 - L.cur;
    void* Sn = h->S[nx];
    void* ASn = h->AS[nx];
    {
      using SU = typename Pol<AU>::S;
      const int c = L.nnow + npn;
      Blk<T> Yn = cat(view<T>(Sn, ld, 0, L.nnow), view<T>(Sn, ld, k, npn));
      if ((AU == Arith::DF64 || AU == Arith::F64) && h->tcU) {
        // tensor-core update: C = [Z(:, :nnow) | C_P] as one float64 s x c
        // matrix (the staging buffer holds smax x (2 k_max + 1) 8-byte values)
        double* Cm = static_cast<double*>(h->Cs);
        {
          Prof p(h, EIG_K_OTHER, 0.0, 0.0);
          CK(cudaMemcpy2DAsync(Cm, sizeof(double) * c, h->Z, sizeof(double) * s, sizeof(double) * L.nnow, s,
                               cudaMemcpyDeviceToDevice, h->st));
          CK(cudaMemcpy2DAsync(Cm + L.nnow, sizeof(double) * c, h->CP, sizeof(double) * npn, sizeof(double) * npn, s,
                               cudaMemcpyDeviceToDevice, h->st));
        }
        if ((rc = o.upd(Sb, Cm, c, c, 1.0, Yn, 0.0))) return rc;
      } else {
        SU* Cs = static_cast<SU*>(h->Cs);
        {
          Prof p(h, EIG_K_OTHER, 0.0, 0.0);
          CK(stage_coef<AU>(s, L.nnow, h->Z, s, Cs, c, 1.0, h->st));
          CK(stage_coef<AU>(s, npn, h->CP, npn, Cs + L.nnow, c, 1.0, h->st));
        }
        const double fl = 2.0 * double(h->n) * s * c, by = Ops<AU, AG>::E * double(h->n) * (s + c);
        Prof p(h, EIG_K_UPDATE, fl, by);
        CK(eig::update<AU>(h->n, Sb, Cs, c, Yn, 0.0, h->st));
      }
      // AX, AP of the new blocks by SpMM (nnz/n is small, so A X costs far
      // less than AS C and keeps AX consistent with X)
      if ((rc = o.spmm(static_cast<T*>(Sn), ld, L.nnow, static_cast<T*>(ASn), ld))) return rc;
      if ((rc = o.spmm(static_cast<T*>(Sn) + k, ld, npn, static_cast<T*>(ASn) + k, ld))) return rc;
    }
    if (debug_on()) {
      o.dbg("new X", view<T>(Sn, ld, 0, L.nnow));
      o.dbg("new P", view<T>(Sn, ld, k, npn));
      o.dbg("C_P (as block)", view<T>(Sn, ld, k, npn));
    }
    L.cur = nx;
    L.np = npn;
    L.poff = 0;
    // shrink: S_drop = [X(:, nes:nnow), P(:, nes-nlock:np)]
    if (L.se.ifshrink(j, L.nnow)) {
      const int hd = h->hdrop;
      const int q = nes - L.nlock;
      CK(cudaMemcpy2DAsync(h->Sd, sizeof(T) * 2 * hd, static_cast<T*>(Sn) + nes, sizeof(T) * ld,
                           sizeof(T) * hd, h->n, cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpy2DAsync(static_cast<T*>(h->Sd) + hd, sizeof(T) * 2 * hd, static_cast<T*>(Sn) + k + q,
                           sizeof(T) * ld, sizeof(T) * hd, h->n, cudaMemcpyDeviceToDevice, h->st));
      L.nnow = nes;
      L.np = q;
      L.have_drop = true;
      if (debug_on()) o.dbg("S_drop at shrink", view<T>(h->Sd, 2 * hd, 0, 2 * hd));
    }
  }
  return EIG_OK;
}

// ---------------------------------------------------------------------------
// Subspace iteration with a Chebyshev filter (Algorithm 1, filter in place
// of the shift-and-invert solve).
// ---------------------------------------------------------------------------
template <Arith AU, Arith AG>
int chebsi_init(eig_handle* h, LState& L) {
  return lobpcg_init<AU, AG>(h, L);  // same set-up: orthogonalise X0, Rayleigh-Ritz
}

template <Arith AU, Arith AG>
int cheb_pre(eig_handle* h, LState& L) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  return o.resid_launch(static_cast<T*>(h->S[L.cur]), static_cast<T*>(h->AS[L.cur]), L.nnow, nullptr, false);
}

template <Arith AU, Arith AG>
int cheb_post(eig_handle* h, LState& L, double switch_r, bool* done, bool* switched) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  const int64_t ld = h->LDS;
  const int k = h->kmax, nes = h->nes;
  *done = false;
  *switched = false;
  int rc;
  {
    const int j = L.j + 1;
    void* Sc = h->S[L.cur];
    void* ASc = h->AS[L.cur];
    T* X = static_cast<T*>(Sc);
    T* AX = static_cast<T*>(ASc);
    ConvInfo ci = conv_test(h, L.nnow);
    if (ci.breakdown) return EIG_EBREAKDOWN;
    h->history.push_back(ci.r);
    L.se.record(j, ci.r, ci.r1);
    L.j = j;
    h->iters = j;
    if (ci.r <= h->opt.tol) {
      *done = true;
      return EIG_OK;
    }
    if (switch_r > 0.0 && ci.r <= switch_r) {
      L.j = j - 1;
      h->history.pop_back();
      L.se.forget(j);
      *switched = true;
      return EIG_OK;
    }
    // filter: Y_m = p_m(A) X, three rotating buffers X, P slot, W slot
    const double* lamh = h->hpin + 2 * h->kmax;
    const double a = lamh[L.nnow - 1], a0 = lamh[0];
    const double b = h->opt.cheb_upper > 0.0 ? h->opt.cheb_upper : h->opt.normA;
    const double e = (b - a) / 2.0, c = (b + a) / 2.0;
    double sigma = e / (a0 - c);
    const double tau = 2.0 / sigma;
    T* bufs[3] = {X, X + k, X + 2 * k};
    // Y1 = (sigma / e) (AX - c X)
    if ((rc = o.axpby_(L.nnow, AX, sigma / e, X, -sigma * c / e, bufs[1]))) return rc;
    int ip = 0, iy = 1;
    for (int d = 2; d <= h->opt.cheb_degree; ++d) {
      const double sn = 1.0 / (tau - sigma);
      const int inew = 3 - ip - iy;
      if ((rc = o.spmm3(bufs[iy], L.nnow, bufs[inew], 2.0 * sn / e, -2.0 * sn * c / e, bufs[ip], -sigma * sn)))
        return rc;
      ip = iy;
      iy = inew;
      sigma = sn;
    }
    // "Powered X_drop": the saved columns get the same filter (no
    // orthogonalisation); temporaries are the two halves of the Wt buffer
    if (h->opt.expand_powered && L.have_drop) {
      const int hd = h->hdrop;
      T* xb[3] = {static_cast<T*>(h->Sd), static_cast<T*>(h->Wt), static_cast<T*>(h->Wt) + hd};
      const int64_t lds[3] = {hd, h->wtw, h->wtw};
      double sg = e / (a0 - c);
      {
        Prof p(h, EIG_K_SPMM, 2.0 * double(h->nnz) * hd, o.spmm_bytes(hd, 2));
        CK(eig::spmm<AU>(o.csr(), hd, xb[0], lds[0], xb[1], lds[1], sg / e, -sg * c / e, nullptr, 0, 0.0, h->st));
      }
      int jp = 0, jy = 1;
      for (int d = 2; d <= h->opt.cheb_degree; ++d) {
        const double sn = 1.0 / (tau - sg);
        const int jn = 3 - jp - jy;
        Prof p(h, EIG_K_SPMM, 2.0 * double(h->nnz) * hd, o.spmm_bytes(hd, 3));
        CK(eig::spmm<AU>(o.csr(), hd, xb[jy], lds[jy], xb[jn], lds[jn], 2.0 * sn / e, -2.0 * sn * c / e, xb[jp],
                         lds[jp], -sg * sn, h->st));
        jp = jy;
        jy = jn;
        sg = sn;
      }
      if (jy != 0)
        CK(cudaMemcpy2DAsync(h->Sd, sizeof(T) * hd, xb[jy], sizeof(T) * lds[jy], sizeof(T) * hd, h->n,
                             cudaMemcpyDeviceToDevice, h->st));
    }
    // expansion: X <- [Y, X_drop]
    Blk<T> Y = view<T>(bufs[iy], ld, 0, L.nnow);
    if (L.se.ifexpand(j, L.nnow)) {
      if (!L.have_drop) return EIG_EINVAL;
      if (h->opt.expand_random)  // 'Random' variant (Sec. 6.4)
        CK(gauss_fill(h->n, h->hdrop, h->Sd, h->hdrop, fmt_of<T>(), h->opt.seed, L.n_exp, h->st));
      ++L.n_exp;
      Y.add(static_cast<T*>(h->Sd), h->hdrop, h->hdrop);
      L.nnow += h->hdrop;
      L.have_drop = false;
    }
    // orthogonalise into the next buffer's X slot, A X, Rayleigh-Ritz
    const int nx = 1 - L.cur;
    void* Sn = h->S[nx];
    void* ASn = h->AS[nx];
    Blk<T> Q;
    Blk<T> Xo = view<T>(Sn, ld, 0, L.nnow);
    Blk<T> mid = view<T>(h->Wt, h->wtw, 0, L.nnow);
    // Y may span two buffers; orth clobbers its source
    if ((rc = o.orth(Q, Y, mid, Xo))) return rc;
    Blk<T> AXo = view<T>(ASn, ld, 0, L.nnow);
    if ((rc = o.spmm_blk(Xo, AXo))) return rc;
    h->widths.push_back(L.nnow);
    if ((rc = o.rr(Xo, AXo))) return rc;
    // X <- X Z back into the current buffer, AX = A X
    if ((rc = o.upd(Xo, h->Z, L.nnow, L.nnow, 1.0, view<T>(Sc, ld, 0, L.nnow), 0.0))) return rc;
    if ((rc = o.spmm(X, ld, L.nnow, AX, ld))) return rc;
    if (L.se.ifshrink(j, L.nnow)) {
      const int hd = h->hdrop;
      CK(cudaMemcpy2DAsync(h->Sd, sizeof(T) * hd, static_cast<T*>(Sc) + nes, sizeof(T) * ld, sizeof(T) * hd,
                           h->n, cudaMemcpyDeviceToDevice, h->st));
      L.nnow = nes;
      L.have_drop = true;
    }
  }
  return EIG_OK;
}

// ---------------------------------------------------------------------------
// Steepest descent with shrink-and-expand (Algorithm 2): Rayleigh-Ritz on
// S = [X, W], W = T R orthogonalised against X; no locking.  On expansion
// X_drop is orthogonalised against X (Algorithm 2 appends it as is, but the
// Rayleigh-Ritz step needs an orthonormal S).
// ---------------------------------------------------------------------------
template <Arith AU, Arith AG>
int sd_post(eig_handle* h, LState& L, double switch_r, bool* done, bool* switched) {
  using T = typename Pol<AU>::T;
  Ops<AU, AG> o(h);
  const int64_t ld = h->LDS;
  const int k = h->kmax, nes = h->nes;
  *done = false;
  *switched = false;
  int rc;
  const int j = L.j + 1;
  void* Sc = h->S[L.cur];
  void* ASc = h->AS[L.cur];
  T* X = static_cast<T*>(Sc);
  T* Wslot = X + 2 * k;
  ConvInfo ci = conv_test(h, L.nnow);
  if (ci.breakdown) return EIG_EBREAKDOWN;
  h->history.push_back(ci.r);
  L.se.record(j, ci.r, ci.r1);
  L.j = j;
  h->iters = j;
  if (ci.r <= h->opt.tol) {
    *done = true;
    return EIG_OK;
  }
  if (switch_r > 0.0 && ci.r <= switch_r) {
    L.j = j - 1;
    h->history.pop_back();
    L.se.forget(j);
    *switched = true;
    return EIG_OK;
  }
  const int nw = L.nnow;  // W = T R has the width of X before any expansion
  if (L.se.ifexpand(j, L.nnow)) {
    if (!L.have_drop) return EIG_EINVAL;
    const int hd = h->hdrop;
    if (h->opt.expand_random)  // 'Random' variant (Sec. 6.4)
      CK(gauss_fill(h->n, hd, h->Sd, hd, fmt_of<T>(), h->opt.seed, L.n_exp, h->st));
    ++L.n_exp;
    Blk<T> Q;
    if (h->opt.deflate_ones) Q.add(FormData<AU>::u0(h), 1, 1);
    Q = cat(Q, view<T>(Sc, ld, 0, L.nnow));
    Blk<T> Dsrc = view<T>(h->Sd, hd, 0, hd);
    Blk<T> Dmid = view<T>(h->Wt, h->wtw, 0, hd);
    Blk<T> Ddst = view<T>(Sc, ld, L.nnow, hd);
    if ((rc = o.orth(Q, Dsrc, Dmid, Ddst))) return rc;
    if ((rc = o.spmm(X + L.nnow, ld, hd, static_cast<T*>(ASc) + L.nnow, ld))) return rc;
    L.nnow += hd;
    L.have_drop = false;
  }
  Blk<T> Xb = view<T>(Sc, ld, 0, L.nnow);
  Blk<T> Q;
  if (h->opt.deflate_ones) Q.add(FormData<AU>::u0(h), 1, 1);
  Q = cat(Q, Xb);
  Blk<T> Wb = view<T>(Sc, ld, 2 * k, nw);
  Blk<T> Wmid = view<T>(h->Wt, h->wtw, 0, nw);
  if ((rc = o.orth(Q, Wb, Wmid, Wb))) return rc;
  if ((rc = o.spmm(Wslot, ld, nw, static_cast<T*>(ASc) + 2 * k, ld))) return rc;
  Blk<T> Sb = cat(Xb, Wb);
  Blk<T> ASb = cat(view<T>(ASc, ld, 0, L.nnow), view<T>(ASc, ld, 2 * k, nw));
  const int s = Sb.width;
  h->widths.push_back(L.nnow);
  if ((rc = o.rr(Sb, ASb))) return rc;
  const int nx = 1 - L.cur;
  void* Sn = h->S[nx];
  void* ASn = h->AS[nx];
  if ((rc = o.upd(Sb, h->Z, s, L.nnow, 1.0, view<T>(Sn, ld, 0, L.nnow), 0.0))) return rc;
  if ((rc = o.spmm(static_cast<T*>(Sn), ld, L.nnow, static_cast<T*>(ASn), ld))) return rc;
  L.cur = nx;
  if (L.se.ifshrink(j, L.nnow)) {
    const int hd = h->hdrop;
    CK(cudaMemcpy2DAsync(h->Sd, sizeof(T) * hd, static_cast<T*>(Sn) + nes, sizeof(T) * ld, sizeof(T) * hd, h->n,
                         cudaMemcpyDeviceToDevice, h->st));
    L.nnow = nes;
    L.have_drop = true;
  }
  return EIG_OK;
}

// Convert the iterate of the float32 phase to double-float storage.
// LOBPCG keeps X, P, AX, AP implicitly consistent, so after the conversion
// [X, P] is re-orthonormalised (the float32 blocks are orthonormal only to
// about 1e-7), AX and AP are recomputed by SpMM and a Rayleigh-Ritz step on X
// restores Ritz vectors; without this the residual would stall near the
// float32 level.
int promote(eig_handle* h, LState& L, int algo) {
  const bool lobpcg = algo == EIG_LOBPCG;
  using T = dd;
  const int64_t ld = h->LDS;
  const int k = h->kmax;
  const int cur = L.cur, nx = 1 - L.cur;
  CK(convert2d(h->n, L.nnow, h->S[cur], ld, EIG_F32, h->S[nx], ld, EIG_DF64, h->st));
  CK(convert2d(h->n, L.nnow, h->AS[cur], ld, EIG_F32, h->AS[nx], ld, EIG_DF64, h->st));
  if (lobpcg && L.np > 0)
    CK(convert2d(h->n, L.np, static_cast<float*>(h->S[cur]) + k + L.poff, ld, EIG_F32,
                 static_cast<dd*>(h->S[nx]) + k, ld, EIG_DF64, h->st));
  if (L.have_drop) {
    const int wd = lobpcg ? 2 * h->hdrop : h->hdrop;
    if (debug_on()) {
      Ops<Arith::F32, Arith::C32> o32(h);
      o32.dbg("S_drop (float) before promotion", view<float>(h->Sd, wd, 0, wd));
    }
    CK(convert2d(h->n, wd, h->Sd, wd, EIG_F32, h->Wt, wd, EIG_DF64, h->st));
    std::swap(h->Sd, h->Wt);
    if (debug_on()) {
      Ops<Arith::DF64, Arith::DF64> o64(h);
      o64.dbg("S_drop (double-float) after promotion", view<dd>(h->Sd, wd, 0, wd));
    }
  }
  L.poff = 0;
  if (algo == EIG_CHEB_SI) {  // re-orthonormalised by the next CholeskyQR2 anyway
    L.cur = nx;
    return EIG_OK;
  }
  Ops<Arith::DF64, Arith::DF64> o(h);
  Blk<T> D = cat(view<T>(h->S[nx], ld, 0, L.nnow), view<T>(h->S[nx], ld, k, L.np));
  Blk<T> mid = view<T>(h->S[cur], ld, 0, L.nnow + L.np);
  Blk<T> Q;
  if (h->opt.deflate_ones) Q.add(h->udd, 1, 1);
  int rc = o.orth(Q, D, mid, D);
  if (rc) return rc;
  Blk<T> X = view<T>(h->S[nx], ld, 0, L.nnow);
  Blk<T> AX = view<T>(h->AS[nx], ld, 0, L.nnow);
  if ((rc = o.spmm_blk(X, AX))) return rc;
  if (L.np > 0 && (rc = o.spmm(static_cast<T*>(h->S[nx]) + k, ld, L.np, static_cast<T*>(h->AS[nx]) + k, ld)))
    return rc;
  if ((rc = o.rr(X, AX))) return rc;
  if ((rc = o.upd(X, h->Z, L.nnow, L.nnow, 1.0, view<T>(h->S[cur], ld, 0, L.nnow), 0.0))) return rc;
  if ((rc = o.spmm(static_cast<T*>(h->S[cur]), ld, L.nnow, static_cast<T*>(h->AS[cur]), ld))) return rc;
  if (L.np > 0) {
    CK(cudaMemcpy2DAsync(static_cast<T*>(h->S[cur]) + k, sizeof(T) * ld, static_cast<T*>(h->S[nx]) + k,
                         sizeof(T) * ld, sizeof(T) * L.np, h->n, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpy2DAsync(static_cast<T*>(h->AS[cur]) + k, sizeof(T) * ld, static_cast<T*>(h->AS[nx]) + k,
                         sizeof(T) * ld, sizeof(T) * L.np, h->n, cudaMemcpyDeviceToDevice, h->st));
  }
  return EIG_OK;
}

// Final float64 pass of every form (the mixed form wins its accuracy back
// here): V = X(:, 1:nev) in float64, orthonormalised by CholeskyQR2 in
// float64, AV = A V by the float64 SpMM, a float64 Rayleigh-Ritz on span(V)
// (V^T A V by the float64 Gram, the float64 eigensolver, V <- V Z and
// AV <- AV Z by the float64 update), and the float64 residual norms of
// Eq. conv with its Ritz values.  All on the CUDA cores in float64; the
// work is n nev^2 per product, once per solve.
int final_pass(eig_handle* h, const void* Xsrc, int src_dt) {
  const int nev = h->nev;
  const int64_t n = h->n;
  double* V = h->V;
  double* tmp = static_cast<double*>(h->Sd);   // n x nev float64 (S_drop is free now)
  double* AV = static_cast<double*>(h->Wt);    // n x nev float64
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int) * NFLAGS, h->st));
  CK(convert2d(n, nev, Xsrc, h->LDS, src_dt, V, nev, EIG_F64, h->st));
  auto blk = [&](double* p) {
    Blk<double> b;
    b.add(p, nev, nev);
    return b;
  };
  // CholeskyQR2: V <- V R^{-1} twice
  for (int pass = 0; pass < 2; ++pass) {
    CK(eig::gram<Arith::F64>(n, blk(V), blk(V), true, h->Gp, nev, h->gscr, h->st));
    CK(chol_rinv(nev, n, h->Gp, nev, h->Rinv, h->cholw, h->flags + F_CHOL1, h->st, nullptr,
                 1.1102230246251565e-16));
    CK(stage_coef<Arith::F64>(nev, nev, h->Rinv, nev, static_cast<double*>(h->Cs), nev, 1.0, h->st));
    CK(eig::update<Arith::F64>(n, blk(V), static_cast<double*>(h->Cs), nev, blk(tmp), 0.0, h->st));
    CK(cudaMemcpyAsync(V, tmp, sizeof(double) * size_t(n) * nev, cudaMemcpyDeviceToDevice, h->st));
  }
  Csr<Arith::F64> c;
  c.n = n;
  c.rowptr = h->rowptr;
  c.colind = h->colind;
  c.val = h->val64;
  c.heavy = h->heavy;
  c.nheavy = h->nheavy;
  c.heavy_min = HEAVY_MIN;
  CK(eig::spmm<Arith::F64>(c, nev, V, nev, AV, nev, 1.0, 0.0, nullptr, 0, 0.0, h->st));
  // Rayleigh-Ritz in float64: V^T A V = Z diag(lam) Z^T, V <- V Z, AV <- AV Z
  CK(eig::gram<Arith::F64>(n, blk(V), blk(AV), true, h->Gp, nev, h->gscr, h->st));
  CK(syev64(nev, h->Gp, nev, h->lamd, h->Z, nev, h->syevw, h->flags + F_SYEV, h->st));
  CK(stage_coef<Arith::F64>(nev, nev, h->Z, nev, static_cast<double*>(h->Cs), nev, 1.0, h->st));
  CK(eig::update<Arith::F64>(n, blk(V), static_cast<double*>(h->Cs), nev, blk(tmp), 0.0, h->st));
  CK(cudaMemcpyAsync(V, tmp, sizeof(double) * size_t(n) * nev, cudaMemcpyDeviceToDevice, h->st));
  CK(eig::update<Arith::F64>(n, blk(AV), static_cast<double*>(h->Cs), nev, blk(tmp), 0.0, h->st));
  CK(eig::residual<Arith::F64>(n, nev, V, nev, tmp, nev, h->lamd, nullptr, nullptr, 0, h->xn, h->rn, h->rscr,
                               h->st));
  std::vector<double> xn(nev), rn(nev), lam(nev);
  int fl[NFLAGS];
  CK(cudaMemcpyAsync(xn.data(), h->xn, sizeof(double) * nev, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(rn.data(), h->rn, sizeof(double) * nev, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(lam.data(), h->lamd, sizeof(double) * nev, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(fl, h->flags, sizeof(fl), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int) * NFLAGS, h->st));
  if (fl[F_CHOL1] == 2 || fl[F_SYEV] != 0) return EIG_EBREAKDOWN;
  h->lam = lam;
  h->resid.resize(nev);
  for (int i = 0; i < nev; ++i) h->resid[i] = std::sqrt(rn[i]) / (h->opt.normA * std::sqrt(xn[i]));
  return EIG_OK;
}

// Resumable solve: init() once, then repeat pre() (launch the residual and
// the copy of its norms), a synchronisation of h->st, and post() (decide and
// launch the rest of the iteration) until finished.  eig_solve runs this
// loop; the serving loop interleaves many of them.
enum Phase { PH_F64 = 0, PH_MIX32 = 1, PH_DF64 = 2 };

struct Stepper {
  eig_handle* h = nullptr;
  LState L;
  int phase = PH_DF64;
  bool lob = true;  // LOBPCG (P block, HL trick); false for subspace iteration and SD
  int algo = EIG_LOBPCG;
  bool finished = false;
  int status = EIG_OK;

  int init() {
    L = LState();
    L.se.kind = h->strategy;
    L.se.nes = h->nes;
    L.se.nex = h->kmax;
    L.se.je = h->opt.je;
    L.se.js = h->opt.js;
    L.se.jp = h->opt.jp;
    L.se.j_warm = h->opt.j_warm;
    L.se.mu = h->opt.mu;
    L.se.r_warm = h->opt.r_warm;
    L.se.warm_first = h->opt.warm_first != 0;
    h->history.clear();
    h->widths.clear();
    h->iters = 0;
    h->n_shrink = h->n_expand = 0;
    std::memset(h->kst, 0, sizeof(h->kst));
    finished = false;
    status = EIG_OK;
    CK(cudaMemsetAsync(h->flags, 0, sizeof(int) * NFLAGS, h->st));
    algo = h->opt.algo;
    lob = algo == EIG_LOBPCG;
    phase = h->opt.form == EIG_FORM_F64 ? PH_F64 : (h->opt.form == EIG_FORM_MIXED ? PH_MIX32 : PH_DF64);
    switch (phase) {
      case PH_F64: return lob ? lobpcg_init<Arith::F64, Arith::F64>(h, L) : chebsi_init<Arith::F64, Arith::F64>(h, L);
      case PH_MIX32: return lob ? lobpcg_init<Arith::F32, Arith::C32>(h, L) : chebsi_init<Arith::F32, Arith::C32>(h, L);
      default: return lob ? lobpcg_init<Arith::DF64, Arith::DF64>(h, L) : chebsi_init<Arith::DF64, Arith::DF64>(h, L);
    }
  }
  // SD writes R into the W slot like LOBPCG, so it shares lob_pre
  int pre() {
    const bool w = algo != EIG_CHEB_SI;
    switch (phase) {
      case PH_F64: return w ? lob_pre<Arith::F64, Arith::F64>(h, L) : cheb_pre<Arith::F64, Arith::F64>(h, L);
      case PH_MIX32: return w ? lob_pre<Arith::F32, Arith::C32>(h, L) : cheb_pre<Arith::F32, Arith::C32>(h, L);
      default: return w ? lob_pre<Arith::DF64, Arith::DF64>(h, L) : cheb_pre<Arith::DF64, Arith::DF64>(h, L);
    }
  }
  int end(int st) {
    h->n_shrink = L.se.n_shrink;
    h->n_expand = L.se.n_expand;
    int frc = final_pass(h, h->S[L.cur], phase == PH_F64 ? EIG_F64 : phase == PH_MIX32 ? EIG_F32 : EIG_DF64);
    finished = true;
    status = frc ? frc : st;
    return status;
  }
  int post() {
    bool done = false, sw = false;
    int rc;
    const double sr = phase == PH_MIX32 ? h->opt.mixed_switch : 0.0;
    switch (phase) {
      case PH_F64:
        rc = algo == EIG_LOBPCG ? lob_post<Arith::F64, Arith::F64>(h, L, sr, &done, &sw)
             : algo == EIG_SD   ? sd_post<Arith::F64, Arith::F64>(h, L, sr, &done, &sw)
                                : cheb_post<Arith::F64, Arith::F64>(h, L, sr, &done, &sw);
        break;
      case PH_MIX32:
        rc = algo == EIG_LOBPCG ? lob_post<Arith::F32, Arith::C32>(h, L, sr, &done, &sw)
             : algo == EIG_SD   ? sd_post<Arith::F32, Arith::C32>(h, L, sr, &done, &sw)
                                : cheb_post<Arith::F32, Arith::C32>(h, L, sr, &done, &sw);
        break;
      default:
        rc = algo == EIG_LOBPCG ? lob_post<Arith::DF64, Arith::DF64>(h, L, sr, &done, &sw)
             : algo == EIG_SD   ? sd_post<Arith::DF64, Arith::DF64>(h, L, sr, &done, &sw)
                                : cheb_post<Arith::DF64, Arith::DF64>(h, L, sr, &done, &sw);
    }
    if (rc) {
      finished = true;
      status = rc;
      return rc;
    }
    const bool out_of_iters = !done && !sw && L.j >= h->opt.max_iter;
    if (phase == PH_MIX32 && (sw || done || out_of_iters)) {
      // promote to double-float storage: the remaining iterations and the
      // final pass read double-float blocks
      if ((rc = promote(h, L, algo))) {
        finished = true;
        status = rc;
        return rc;
      }
      phase = PH_DF64;
      if (sw) return EIG_OK;
    }
    if (done) return end(EIG_OK);
    if (out_of_iters) return end(EIG_ENOTCONV);
    return EIG_OK;
  }
};

int solve_impl(eig_handle* h) {
  Stepper st;
  st.h = h;
  int rc = st.init();
  if (rc) return rc;
  while (!st.finished) {
    if ((rc = st.pre())) return rc;
    CK(cudaStreamSynchronize(h->st));
    prof_flush(h);
    st.post();
  }
  return st.status;
}

void free_all(eig_handle* h) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  if (h->own_idx) {
    F(h->rowptr);
    F(h->colind);
  }
  F(h->heavy);
  F(h->val64);
  F(h->valdd);
  F(h->val32);
  F(h->t64);
  F(h->tdd);
  F(h->t32);
  F(h->u64);
  F(h->udd);
  F(h->u32);
  F(h->S[0]);
  F(h->S[1]);
  F(h->AS[0]);
  F(h->AS[1]);
  F(h->Wt);
  F(h->Sd);
  F(h->tcU);
  F(h->tcV);
  F(h->tcC);
  F(h->tcQc);
  F(h->tcQr);
  F(h->Gt);
  F(h->Gp);
  F(h->Rinv);
  F(h->cholw);
  F(h->Z);
  F(h->lamd);
  F(h->CP);
  F(h->gscr);
  F(h->rscr);
  F(h->xn);
  F(h->rn);
  F(h->Cs);
  F(h->syevw);
  F(h->hlw);
  F(h->flags);
  F(h->V);
  if (h->hpin) cudaFreeHost(h->hpin);
}

__global__ void diag_inv_kernel(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* val,
                                double* t) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
    if (colind[q] == i) d += val[q];
  t[i] = d != 0.0 ? 1.0 / d : 1.0;
}

__global__ void fill_kernel(int64_t n, double v, double* x) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

}  // namespace

// Device bytes eig_create allocates (same formulas as its allocations).
size_t footprint_bytes(int64_t n, int64_t nnz, int nev, int k_max, int nes, int form, int precond,
                       int deflate, int on_device, int gram_tc, int tc_chunk_rows) {
  const size_t LDS = size_t((3 * k_max + 3) / 4 * 4);
  const size_t hd = size_t(k_max - nes);
  const size_t wtw = std::max(size_t(k_max), 2 * hd);
  const size_t cq = std::max(wtw, size_t(2 * k_max));
  const size_t smax = size_t(3 * k_max + 1);
  size_t b = 0;
  if (!on_device) b += 4 * size_t(n + 1) + 4 * size_t(nnz);
  b += 8 * size_t(nnz) * 2;                      // float64 + double-float values
  if (form == EIG_FORM_MIXED) b += 4 * size_t(nnz);
  if (precond) b += 20 * size_t(n);
  if (deflate) b += 20 * size_t(n);
  b += 4 * 8 * size_t(n) * LDS;                  // S, AS (two copies each)
  b += 2 * 8 * size_t(n) * std::max(wtw, size_t(nev));
  b += 8 * size_t(n) * nev;                      // V
  b += 8 * (smax * smax * 2 + cq * cq * 2 + 2 * cq + smax * k_max + smax * (2 * k_max + 1) + 4 * smax);
  b += 8 * (size_t(2) * num_sms() * 4 * 64 * 64 + smax * smax + 4096);
  b += 8 * residual_scratch_elems(n, k_max);
  b += std::max(syev_work_bytes(int(smax)), syev64_work_bytes(int(smax))) + hl_work_bytes(int(smax), k_max, 0) +
       8 * smax * smax;
  if (gram_tc) {
    const int ns = tc_slices(form);
    const int64_t rows = tc_rows_of(n, tc_chunk_rows);
    b += 2 * tc_operand_bytes(ns, rows, int(smax)) + tc_slice_bytes(ns, int64_t(smax), 2 * k_max + 1);
    if (rows == n)
      b += 2 * tc_operand_bytes(ns, n, 2 * k_max + 1);   // slices of [u0, X, P], both layouts
    else
      b += 8 * smax * smax;                              // Gram of one row chunk
  }
  return b + b / 16 + (size_t(32) << 20);        // allocator rounding and slack
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* eig_strerror(int s) {
  switch (s) {
    case EIG_OK: return "ok";
    case EIG_EINVAL: return "invalid argument";
    case EIG_ENOMEM: return "out of device memory";
    case EIG_ENOTCONV: return "not converged within max_iter";
    case EIG_EBREAKDOWN: return "orthogonalisation or eigensolver breakdown";
    case EIG_ECUDA: return "CUDA error";
    case EIG_ETIMEOUT: return "bounded device wait expired";
    case EIG_EBUSY: return "no free serving slot";
    case EIG_EREJECT: return "request can never fit";
    default: return "unknown status";
  }
}

int eig_options_default(eig_options* o) {
  if (!o) return EIG_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->algo = EIG_LOBPCG;
  o->form = EIG_FORM_F64;
  o->tol = 1e-10;
  o->max_iter = 1000;
  o->nes = 0;
  o->je = 12;
  o->js = 2;
  o->jp = 10;
  o->j_warm = 5;
  o->mu = 1.1;
  o->r_warm = 1e-4;
  o->cheb_degree = 12;
  o->cheb_upper = 0.0;
  o->precond = 0;
  o->deflate_ones = 0;
  o->normA = 0.0;
  o->mixed_switch = 1e-5;
  o->gram_tc = 1;
  return EIG_OK;
}

int eig_strategy_trace(int strategy, int nes, int nex, const eig_options* opt, const double* r, const double* r1,
                       int m, int* width, int* events, int max_events, int* n_events) {
  if (strategy < EIG_NONE || strategy > EIG_SLOPEK || nes < 1 || nes >= nex || m < 0 || max_events < 0 ||
      !n_events || (m > 0 && !r) || (max_events > 0 && !events))
    return EIG_EINVAL;
  eig_options d;
  eig_options_default(&d);
  const eig_options* o = opt ? opt : &d;
  SEStrategy se;
  se.kind = strategy;
  se.nes = nes;
  se.nex = nex;
  se.je = o->je;
  se.js = o->js;
  se.jp = o->jp;
  se.j_warm = o->j_warm;
  se.mu = o->mu;
  se.r_warm = o->r_warm;
  se.warm_first = o->warm_first != 0;
  if (se.je < 1 || se.js < 1 || se.jp < 1) return EIG_EINVAL;
  int nnow = nex, ne = 0;
  auto event = [&](int j, int kind) {
    if (ne < max_events) {
      events[2 * ne] = j;
      events[2 * ne + 1] = kind;
    }
    ++ne;
  };
  // the order of the decision points in an iteration of eig_solve
  for (int j = 1; j <= m; ++j) {
    const double rf = r1 ? r1[j - 1] : r[j - 1];
    if (!(r[j - 1] >= 0.0) || !(rf >= 0.0)) return EIG_EINVAL;
    se.record(j, r[j - 1], rf);
    if (se.ifexpand(j, nnow)) {
      nnow = nex;
      event(j, EIG_EVENT_EXPAND);
    }
    if (width) width[j - 1] = nnow;
    if (se.ifshrink(j, nnow)) {
      nnow = nes;
      event(j, EIG_EVENT_SHRINK);
    }
  }
  *n_events = ne;
  return EIG_OK;
}

int eig_create(const eig_csr* A, int nev, int k_max, int strategy, const eig_options* opt, eig_handle** out) {
  if (!A || !out || !opt) return EIG_EINVAL;
  *out = nullptr;
  const int nes = opt->nes > 0 ? opt->nes : nev + 5;
  if (A->n <= 0 || A->nnz < 0 || !A->rowptr || !A->colind || !A->val) return EIG_EINVAL;
  if (A->val_dtype != EIG_F64 && A->val_dtype != EIG_F32) return EIG_EINVAL;
  if (nev < 1 || nes < nev || nes >= k_max || k_max > A->n) return EIG_EINVAL;
  if (strategy < EIG_NONE || strategy > EIG_SLOPEK) return EIG_EINVAL;
  if (!opt->X0 || !(opt->normA >= 0.0) || opt->max_iter < 1 || !(opt->tol > 0.0)) return EIG_EINVAL;
  if (opt->algo != EIG_LOBPCG && opt->algo != EIG_CHEB_SI && opt->algo != EIG_SD) return EIG_EINVAL;
  if (opt->form < EIG_FORM_DF64 || opt->form > EIG_FORM_MIXED) return EIG_EINVAL;
  if (opt->algo == EIG_CHEB_SI && opt->cheb_degree < 2) return EIG_EINVAL;
  if (opt->je < 1 || opt->js < 0 || opt->jp < 1) return EIG_EINVAL;
  if (opt->expand_random != 0 && opt->expand_random != 1) return EIG_EINVAL;
  if (opt->expand_random && opt->expand_powered) return EIG_EINVAL;
  if (opt->tc_chunk_rows < 0 || opt->tc_chunk_rows % 128 != 0) return EIG_EINVAL;
  if (k_max > 1400) return EIG_EINVAL;
  eig_handle* h = new eig_handle();
  h->n = A->n;
  h->nnz = A->nnz;
  h->nev = nev;
  h->kmax = k_max;
  h->nes = nes;
  h->strategy = strategy;
  h->opt = *opt;
  h->opt.nes = nes;
  h->st = static_cast<cudaStream_t>(opt->stream);
  h->LDS = ((3 * k_max) + 3) / 4 * 4;
  h->hdrop = k_max - nes;
  h->wtw = std::max(k_max, 2 * h->hdrop);
  const int64_t n = A->n, nnz = A->nnz;
  auto fail = [&](int code) {
    free_all(h);
    delete h;
    return code;
  };
#define AL(ptr, bytes)                                                            \
  do {                                                                            \
    if (cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 16) != cudaSuccess) {  \
      cudaGetLastError();                                                         \
      return fail(EIG_ENOMEM);                                                    \
    }                                                                             \
  } while (0)
  // CSR; float32 values are staged in val32 and widened into val64
  const bool v32 = A->val_dtype == EIG_F32;
  void* vdst = nullptr;
  if (v32) {
    AL(h->val32, sizeof(float) * nnz);
    vdst = h->val32;
  }
  AL(h->val64, sizeof(double) * nnz);
  if (!v32) vdst = h->val64;
  const size_t vbytes = (v32 ? sizeof(float) : sizeof(double)) * nnz;
  if (A->on_device) {
    h->rowptr = const_cast<int32_t*>(A->rowptr);
    h->colind = const_cast<int32_t*>(A->colind);
    if (cudaMemcpyAsync(vdst, A->val, vbytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess)
      return fail(EIG_ECUDA);
  } else {
    h->own_idx = true;
    AL(h->rowptr, sizeof(int32_t) * (n + 1));
    AL(h->colind, sizeof(int32_t) * nnz);
    if (cudaMemcpyAsync(h->rowptr, A->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, h->st) ||
        cudaMemcpyAsync(h->colind, A->colind, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, h->st) ||
        cudaMemcpyAsync(vdst, A->val, vbytes, cudaMemcpyHostToDevice, h->st))
      return fail(EIG_ECUDA);
  }
  if (v32 && convert2d(1, nnz, h->val32, nnz, EIG_F32, h->val64, nnz, EIG_F64, h->st)) return fail(EIG_ECUDA);
  {
    // power-law rows for the split SpMM path (read from the host copy of
    // rowptr, or once from the device)
    std::vector<int32_t> rp;
    const int32_t* hrp = A->rowptr;
    if (A->on_device) {
      rp.resize(size_t(n) + 1);
      if (cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, h->st) ||
          cudaStreamSynchronize(h->st))
        return fail(EIG_ECUDA);
      hrp = rp.data();
    }
    std::vector<int32_t> hv;
    for (int64_t i = 0; i < n; ++i)
      if (hrp[i + 1] - hrp[i] > HEAVY_MIN) hv.push_back(int32_t(i));
    if (opt->normA == 0.0) {  // ||A||_2 of Eq. conv not given: the Gershgorin bound
      const void* hval = A->val;
      std::vector<double> vbuf;
      if (A->on_device) {
        const size_t vb = (A->val_dtype == EIG_F32 ? sizeof(float) : sizeof(double)) * size_t(nnz);
        vbuf.resize((vb + sizeof(double) - 1) / sizeof(double));
        if (cudaMemcpyAsync(vbuf.data(), A->val, vb, cudaMemcpyDeviceToHost, h->st) ||
            cudaStreamSynchronize(h->st))
          return fail(EIG_ECUDA);
        hval = vbuf.data();
      }
      h->opt.normA = gershgorin_bound(n, hrp, hval, A->val_dtype);
      if (!(h->opt.normA > 0.0)) return fail(EIG_EINVAL);  // the zero matrix
    }
    if (!hv.empty()) {
      AL(h->heavy, sizeof(int32_t) * hv.size());
      if (cudaMemcpyAsync(h->heavy, hv.data(), sizeof(int32_t) * hv.size(), cudaMemcpyHostToDevice, h->st) ||
          cudaStreamSynchronize(h->st))
        return fail(EIG_ECUDA);
      h->nheavy = int(hv.size());
    }
  }
  AL(h->valdd, sizeof(dd) * nnz);
  if (convert2d(1, nnz, h->val64, nnz, EIG_F64, h->valdd, nnz, EIG_DF64, h->st)) return fail(EIG_ECUDA);
  if (opt->form == EIG_FORM_MIXED && !v32) {
    AL(h->val32, sizeof(float) * nnz);
    if (convert2d(1, nnz, h->val64, nnz, EIG_F64, h->val32, nnz, EIG_F32, h->st)) return fail(EIG_ECUDA);
  } else if (opt->form != EIG_FORM_MIXED && v32) {
    // the float32 staging copy is not part of the handle's footprint
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(EIG_ECUDA);
    cudaFree(h->val32);
    h->val32 = nullptr;
  }
  if (opt->precond) {
    AL(h->t64, sizeof(double) * n);
    AL(h->tdd, sizeof(dd) * n);
    AL(h->t32, sizeof(float) * n);
    diag_inv_kernel<<<(unsigned)cdiv(n, 256), 256, 0, h->st>>>(n, h->rowptr, h->colind, h->val64, h->t64);
    convert2d(1, n, h->t64, n, EIG_F64, h->tdd, n, EIG_DF64, h->st);
    convert2d(1, n, h->t64, n, EIG_F64, h->t32, n, EIG_F32, h->st);
  }
  if (opt->deflate_ones) {
    AL(h->u64, sizeof(double) * n);
    AL(h->udd, sizeof(dd) * n);
    AL(h->u32, sizeof(float) * n);
    fill_kernel<<<(unsigned)cdiv(n, 256), 256, 0, h->st>>>(n, 1.0 / std::sqrt(double(n)), h->u64);
    convert2d(1, n, h->u64, n, EIG_F64, h->udd, n, EIG_DF64, h->st);
    convert2d(1, n, h->u64, n, EIG_F64, h->u32, n, EIG_F32, h->st);
  }
  // blocks
  const size_t blk = sizeof(double) * size_t(n) * h->LDS;
  AL(h->S[0], blk);
  AL(h->S[1], blk);
  AL(h->AS[0], blk);
  AL(h->AS[1], blk);
  AL(h->Wt, sizeof(double) * size_t(n) * std::max(h->wtw, nev));
  // S_drop and Wt are swapped when the mixed form promotes; same size
  AL(h->Sd, sizeof(double) * size_t(n) * std::max(h->wtw, nev));
  if (uses_gram_tc(h->opt)) {
    const int ns = h->tcns = tc_slices(opt->form);
    h->tcrows = tc_rows_of(n, opt->tc_chunk_rows);
    AL(h->tcU, tc_operand_bytes(ns, h->tcrows, 3 * k_max + 1));
    AL(h->tcV, tc_operand_bytes(ns, h->tcrows, 3 * k_max + 1));
    AL(h->tcC, tc_slice_bytes(ns, 3 * k_max + 1, 2 * k_max + 1));
    if (h->tcrows == n) {
      h->qcmax = 2 * k_max + 1;  // [u0, X, P]
      AL(h->tcQc, tc_operand_bytes(ns, n, h->qcmax));
      AL(h->tcQr, tc_operand_bytes(ns, n, h->qcmax));
    } else {
      AL(h->Gt, sizeof(double) * size_t(3 * k_max + 1) * (3 * k_max + 1));
    }
  }
  // small
  const int smax = 3 * k_max + 1;
  h->smax = smax;
  AL(h->Gp, sizeof(double) * size_t(smax) * smax);
  // CholeskyQR widths: W (<= k_max), S_drop (2 (k_max - nes)) and, when the
  // mixed form promotes, [X, P] (<= 2 k_max)
  h->cqmax = std::max(h->wtw, 2 * k_max);
  AL(h->Rinv, sizeof(double) * size_t(h->cqmax) * h->cqmax);
  AL(h->cholw, sizeof(double) * (size_t(h->cqmax) * h->cqmax + 2 * size_t(h->cqmax)));
  AL(h->Z, sizeof(double) * size_t(smax) * smax);
  AL(h->lamd, sizeof(double) * smax);
  AL(h->CP, sizeof(double) * size_t(smax) * k_max);
  const size_t gs = size_t(2) * num_sms() * 4 * 64 * 64 + size_t(smax) * smax + 4096;
  AL(h->gscr, sizeof(double) * gs);
  AL(h->rscr, sizeof(double) * residual_scratch_elems(n, k_max));
  AL(h->xn, sizeof(double) * smax);
  AL(h->rn, sizeof(double) * smax);
  AL(h->Cs, sizeof(double) * size_t(smax) * (2 * k_max + 1));
  AL(h->syevw, std::max(syev_work_bytes(smax), syev64_work_bytes(smax)));
  AL(h->hlw, hl_work_bytes(smax, k_max, 0) + sizeof(double) * size_t(smax) * smax);
  AL(h->flags, sizeof(int) * NFLAGS);
  AL(h->V, sizeof(double) * size_t(n) * nev);
  if (cudaMallocHost((void**)&h->hpin, sizeof(double) * (3 * size_t(k_max) + 16)) != cudaSuccess)
    return fail(EIG_ENOMEM);
#undef AL
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(EIG_ECUDA);
  *out = h;
  return EIG_OK;
}

int eig_solve(eig_handle* h) {
  if (!h) return EIG_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launches_total();
  int rc = solve_impl(h);
  cudaStreamSynchronize(h->st);
  if (h->tcU) {  // a bounded wait of a tensor-core product ran out
    const int v = tc::tc5_take_error();
    if (v != 0 && rc == EIG_OK) rc = v > 0 ? EIG_ETIMEOUT : EIG_ECUDA;
  }
  prof_flush(h);
  auto t1 = std::chrono::steady_clock::now();
  h->time_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  h->launches = launches_total() - l0;
  h->status = rc;
  return rc;
}

int eig_query(const eig_handle* h, eig_result* out) {
  if (!h || !out) return EIG_EINVAL;
  out->status = h->status;
  out->iters = h->iters;
  out->n_shrink = h->n_shrink;
  out->n_expand = h->n_expand;
  out->nev = h->nev;
  out->lambda = h->lam.empty() ? nullptr : h->lam.data();
  out->resid = h->resid.empty() ? nullptr : h->resid.data();
  out->V = h->V;
  out->history = h->history.empty() ? nullptr : h->history.data();
  out->widths = h->widths.empty() ? nullptr : h->widths.data();
  out->time_ms = h->time_ms;
  out->normA = h->opt.normA;
  out->kstats = &h->kst[0][0];
  out->launches = h->launches;
  return EIG_OK;
}

void eig_destroy(eig_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  prof_flush(h);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  free_all(h);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: a request loop over independent solves.  eig_submit queues a
// request (host data copied); eig_server_step admits queued requests in
// arrival order while their device footprint fits the memory budget and a
// slot is free, then advances every active solve by one iteration: first the
// residual and norm copy of every solve is launched on its own stream, then
// each stream is synchronised in turn and its decisions taken and the rest of
// its iteration launched, so the solves' kernels overlap on the device and
// each takes its shrink / expand decisions independently.  A finished solve
// copies its results to host memory, frees its device memory and its slot.
// ---------------------------------------------------------------------------
namespace {

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> rowptr, colind;
  std::vector<double> val, X0;
  int nev = 0, k_max = 0, strategy = 0;
  eig_options opt{};
  size_t footprint = 0;
  std::chrono::steady_clock::time_point t_submit, t_done;
  // active state
  eig_handle* h = nullptr;
  cudaStream_t st = nullptr;
  Stepper stp;
  // results
  bool done = false;
  int status = EIG_OK;
  int iters = 0, n_shrink = 0, n_expand = 0;
  std::vector<double> lam, resid, history, V;
  std::vector<int> widths;
};

}  // namespace

struct eig_server {
  eig_server_opts opt{};
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  std::vector<Request*> queue, active;
  std::vector<Request*> finished;
  ~eig_server() {
    for (auto* r : queue) delete r;
    for (auto* r : active) {
      if (r->h) eig_destroy(r->h);
      if (r->st) cudaStreamDestroy(r->st);
      delete r;
    }
    for (auto* r : finished) delete r;
  }
};

namespace {

Request* find_req(eig_server* s, uint64_t t) {
  for (auto* r : s->finished)
    if (r->ticket == t) return r;
  for (auto* r : s->active)
    if (r->ticket == t) return r;
  for (auto* r : s->queue)
    if (r->ticket == t) return r;
  return nullptr;
}

int admit(eig_server* s, Request* r) {
  if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) return EIG_ECUDA;
  eig_csr A{r->n, r->nnz, r->rowptr.data(), r->colind.data(), r->val.data(), 0, EIG_F64};
  eig_options o = r->opt;
  o.X0 = r->X0.data();
  o.x0_on_device = 0;
  o.stream = r->st;
  int rc = eig_create(&A, r->nev, r->k_max, r->strategy, &o, &r->h);
  if (rc) return rc;
  r->stp = Stepper();
  r->stp.h = r->h;
  rc = r->stp.init();
  if (rc) return rc;
  s->in_use += r->footprint;
  return EIG_OK;
}

void retire(eig_server* s, Request* r) {
  eig_handle* h = r->h;
  r->status = r->stp.status;
  r->iters = h->iters;
  r->n_shrink = h->n_shrink;
  r->n_expand = h->n_expand;
  r->lam = h->lam;
  r->resid = h->resid;
  r->history = h->history;
  r->widths = h->widths;
  r->opt.normA = h->opt.normA;  // the Gershgorin bound when the request left it 0
  r->V.resize(size_t(r->n) * r->nev);
  if (r->status == EIG_OK || r->status == EIG_ENOTCONV)
    cudaMemcpyAsync(r->V.data(), h->V, sizeof(double) * r->V.size(), cudaMemcpyDeviceToHost, r->st);
  cudaStreamSynchronize(r->st);
  r->t_done = std::chrono::steady_clock::now();
  r->done = true;
  eig_destroy(h);
  r->h = nullptr;
  cudaStreamDestroy(r->st);
  r->st = nullptr;
  s->in_use -= std::min(s->in_use, r->footprint);
  r->rowptr.clear();
  r->colind.clear();
  r->val.clear();
  r->X0.clear();
}

}  // namespace

extern "C" {

int eig_norm_bound(const eig_csr* A, double* out) {
  if (!A || !out || A->on_device || A->n <= 0 || !A->rowptr || !A->val) return EIG_EINVAL;
  if (A->val_dtype != EIG_F64 && A->val_dtype != EIG_F32) return EIG_EINVAL;
  if (A->rowptr[0] != 0) return EIG_EINVAL;
  for (int64_t i = 0; i < A->n; ++i)
    if (A->rowptr[i + 1] < A->rowptr[i]) return EIG_EINVAL;
  *out = gershgorin_bound(A->n, A->rowptr, A->val, A->val_dtype);
  return EIG_OK;
}

size_t eig_footprint(int64_t n, int64_t nnz, int nev, int k_max, const eig_options* opt) {
  eig_options d;
  eig_options_default(&d);
  const eig_options* o = opt ? opt : &d;
  const int nes = o->nes > 0 ? o->nes : nev + 5;
  return footprint_bytes(n, nnz, nev, k_max, nes, o->form, o->precond, o->deflate_ones, 0, o->gram_tc,
                         o->tc_chunk_rows);
}

int eig_server_create(const eig_server_opts* opts, eig_server** out) {
  if (!opts || !out || opts->mem_budget_bytes == 0 || opts->max_active < 1) return EIG_EINVAL;
  eig_server* s = new eig_server();
  s->opt = *opts;
  *out = s;
  return EIG_OK;
}

int eig_submit(eig_server* s, const eig_csr* A, int nev, int k_max, int strategy, const eig_options* opt,
               uint64_t* ticket) {
  if (!s || !A || !opt || !ticket || A->on_device || !opt->X0 || opt->x0_on_device) return EIG_EINVAL;
  if (A->val_dtype != EIG_F64 && A->val_dtype != EIG_F32) return EIG_EINVAL;
  const int nes = opt->nes > 0 ? opt->nes : nev + 5;
  if (A->n <= 0 || nev < 1 || nes < nev || nes >= k_max || k_max > A->n || !(opt->normA >= 0.0)) return EIG_EINVAL;
  Request* r = new Request();
  r->ticket = s->next_ticket++;
  r->n = A->n;
  r->nnz = A->nnz;
  r->rowptr.assign(A->rowptr, A->rowptr + A->n + 1);
  r->colind.assign(A->colind, A->colind + A->nnz);
  if (A->val_dtype == EIG_F32) {
    const float* v = static_cast<const float*>(A->val);
    r->val.assign(v, v + A->nnz);
  } else {
    const double* v = static_cast<const double*>(A->val);
    r->val.assign(v, v + A->nnz);
  }
  r->X0.assign(opt->X0, opt->X0 + size_t(A->n) * k_max);
  r->nev = nev;
  r->k_max = k_max;
  r->strategy = strategy;
  r->opt = *opt;
  r->footprint = footprint_bytes(A->n, A->nnz, nev, k_max, nes, opt->form, opt->precond, opt->deflate_ones, 0,
                                 opt->gram_tc, opt->tc_chunk_rows);
  r->t_submit = std::chrono::steady_clock::now();
  if (r->footprint > s->opt.mem_budget_bytes) {
    delete r;
    return EIG_EREJECT;
  }
  s->queue.push_back(r);
  *ticket = r->ticket;
  return EIG_OK;
}

int eig_server_step(eig_server* s, int* n_active, int* n_queued) {
  if (!s) return EIG_EINVAL;
  std::vector<Request*> pending;
  // the device part of r's next iteration, up to the copy of its residual
  // norms
  auto launch_one = [&](Request* r) {
    int rc = r->stp.pre();
    if (rc) {
      r->stp.finished = true;
      r->stp.status = rc;
    }
    pending.push_back(r);
  };
  // admission in arrival order; an admitted solve launches its first
  // iteration at once
  auto admit_queued = [&]() {
    while (!s->queue.empty() && int(s->active.size()) < s->opt.max_active &&
           s->in_use + s->queue.front()->footprint <= s->opt.mem_budget_bytes) {
      Request* r = s->queue.front();
      s->queue.erase(s->queue.begin());
      int rc = admit(s, r);
      if (rc) {
        r->status = rc;
        r->done = true;
        r->t_done = std::chrono::steady_clock::now();
        if (r->h) eig_destroy(r->h);
        if (r->st) cudaStreamDestroy(r->st);
        r->h = nullptr;
        r->st = nullptr;
        s->finished.push_back(r);
        continue;
      }
      s->active.push_back(r);
      launch_one(r);
    }
  };
  for (auto* r : s->active) launch_one(r);
  admit_queued();
  // every active solve advances by one iteration; the host part of each
  // (strategy decision, small eigenproblems launched, bookkeeping) runs as
  // soon as its own stream has drained, in completion order, so that a
  // short iteration does not wait behind a long one; a finished solve frees
  // its slot and memory at once and the queue is admitted into it
  while (!pending.empty()) {
    bool progressed = false;
    for (size_t i = 0; i < pending.size();) {
      Request* r = pending[i];
      if (!r->stp.finished) {
        const cudaError_t q = cudaStreamQuery(r->st);
        if (q == cudaErrorNotReady) {
          ++i;
          continue;
        }
        if (q != cudaSuccess) {
          cudaGetLastError();
          r->stp.finished = true;
          r->stp.status = EIG_ECUDA;
        } else {
          prof_flush(r->h);
          r->stp.post();
        }
      }
      progressed = true;
      pending.erase(pending.begin() + i);
      if (r->stp.finished) {
        retire(s, r);
        s->finished.push_back(r);
        s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        admit_queued();
      }
    }
    if (!progressed) std::this_thread::yield();
  }
  if (n_active) *n_active = int(s->active.size());
  if (n_queued) *n_queued = int(s->queue.size());
  return EIG_OK;
}

int eig_poll(eig_server* s, uint64_t ticket, eig_result* out, int* ready) {
  if (!s || !out || !ready) return EIG_EINVAL;
  Request* r = find_req(s, ticket);
  if (!r) return EIG_EINVAL;
  *ready = r->done ? 1 : 0;
  std::memset(out, 0, sizeof(*out));
  if (!r->done) return EIG_OK;
  out->status = r->status;
  out->iters = r->iters;
  out->n_shrink = r->n_shrink;
  out->n_expand = r->n_expand;
  out->nev = r->nev;
  out->lambda = r->lam.empty() ? nullptr : r->lam.data();
  out->resid = r->resid.empty() ? nullptr : r->resid.data();
  out->V = r->V.empty() ? nullptr : r->V.data();
  out->history = r->history.empty() ? nullptr : r->history.data();
  out->widths = r->widths.empty() ? nullptr : r->widths.data();
  out->time_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  out->normA = r->opt.normA;
  return EIG_OK;
}

int eig_release(eig_server* s, uint64_t ticket) {
  if (!s) return EIG_EINVAL;
  for (size_t i = 0; i < s->finished.size(); ++i)
    if (s->finished[i]->ticket == ticket) {
      delete s->finished[i];
      s->finished.erase(s->finished.begin() + i);
      return EIG_OK;
    }
  return EIG_EINVAL;
}

void eig_server_destroy(eig_server* s) { delete s; }

}  // extern "C"
