/*
 * eig_gb300.h -- C ABI of the GB300-native shrink-and-expand block
 * eigensolvers (Liu, Ma and Shao, "On a shrink-and-expand technique for
 * symmetric block eigensolvers", arXiv:2409.05572).
 *
 * Problem (Sec. 1): for a sparse symmetric A (n x n), find the nev
 * algebraically smallest eigenpairs A V = V Lambda.  Method: LOBPCG with
 * soft locking (Algorithm 3) or subspace iteration with a Chebyshev filter in
 * place of the shift-and-invert solve (Algorithm 1), inside the shrink-and-
 * expand framework (Algorithm 5) driven by the fix / slope / slopek strategies
 * (Algorithms 6 and 7) after a warm-up (end of Sec. 3.2).
 *
 * Conventions for every entry point:
 *  - Return value: an EIG_* status; 0 is success.  eig_strerror() names it.
 *    On EIG_EINVAL nothing was launched.  On EIG_ECUDA a CUDA call failed;
 *    the sticky CUDA error state, if any, is left as CUDA set it.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are ordinary process memory.  The library never
 *    frees memory it did not allocate.
 *  - Blocks are row-major: element (i, j) of an n x w block with leading
 *    dimension ld (in elements, ld >= w) is at p[i*ld + j].
 *  - Element formats (dtype): EIG_F64 float64; EIG_F32 float32; EIG_DF64
 *    "double-float": each element is a pair {float hi, float lo} (8 bytes,
 *    value hi + lo, |lo| <= ulp(hi)/2), the block format of the double-float
 *    form, whose block arithmetic runs on the FP32 pipes.
 *  - stream: a cudaStream_t (NULL = legacy default stream).  Low-level
 *    kernels are asynchronous on it; eig_solve() blocks until the solve ends.
 *  - Low-level entry points allocate their temporary device memory with
 *    cudaMallocAsync/cudaFreeAsync on the given stream.
 */
#ifndef EIG_GB300_H
#define EIG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define EIG_OK 0
#define EIG_EINVAL 1      /* bad argument (sizes, pointers, options)          */
#define EIG_ENOMEM 2      /* device allocation failed                         */
#define EIG_ENOTCONV 3    /* max_iter reached; partial results queryable      */
#define EIG_EBREAKDOWN 4  /* orthogonalisation lost rank beyond recovery      */
#define EIG_ECUDA 5       /* a CUDA runtime call failed                       */
#define EIG_ETIMEOUT 6    /* a bounded device wait expired                    */
#define EIG_EBUSY 7       /* serving: no free slot                            */
#define EIG_EREJECT 8     /* serving: request can never fit                   */

/* ---- element formats and arithmetic ----------------------------------- */
#define EIG_F64 0
#define EIG_F32 1
#define EIG_DF64 2

/* arithmetic of the block kernels (SpMM, Gram, update, residual)          */
#define EIG_ARITH_F64 0   /* float64 blocks, native FP64 FMA                 */
#define EIG_ARITH_DF64 1  /* double-float blocks, FP32-pipe dd arithmetic    */
#define EIG_ARITH_F32 2   /* float32 blocks, float32 arithmetic              */
#define EIG_ARITH_C32 3   /* float32 blocks, compensated (Dot2) accumulation */
/* eig_gram and eig_block_update only: products on the bf16 tensor cores by
 * an exact integer splitting (Ozaki et al. 2012).  Each value is cut into
 * 8-bit slices against a power-of-two scale shared by a 128-index chunk of
 * the contraction (128 rows of a column of U or V for the Gram; 128 columns
 * of a row of U and 128 rows of a column of C for the update); the slice
 * products of the kept levels are summed exactly in fp32 and the rest
 * dropped.  The error is normwise: a bound per contraction index of a
 * multiple of the product of the two chunk maxima.
 *  EIG_ARITH_DF64_TC: EIG_DF64 blocks, six slices, levels 0..5: at most about
 *    28 * 2^-48 of the chunk maxima per index (about 2^-48 on average),
 *    double-float result; chunks whose maximum is below 2^-100 count as zero.
 *  EIG_ARITH_F64_TC: EIG_F64 blocks, seven slices cut from the float64 bit
 *    patterns by integer operations, levels 0..6, accumulated in
 *    triple-float: at most about 2^-52 of the chunk maxima per index plus
 *    2^-53 of the chunk sums per chunk -- the float64 dot-product bound with
 *    the chunk maxima in place of the elements.  Subnormal values count as
 *    zero; an infinite or NaN value makes the entries it touches NaN. */
#define EIG_ARITH_DF64_TC 4
#define EIG_ARITH_F64_TC 5

/* ---- conversions ------------------------------------------------------- */
/* dst[i] = src[i] for i < count, converting between EIG_F64 / EIG_F32 /
 * EIG_DF64 elements (device pointers; src and dst must not overlap). */
int eig_convert(int64_t count, const void *src, int src_dtype, void *dst, int dst_dtype,
                void *stream);

/* ---- a7 / a13: sparse block product (Algorithms 1-3: A X, A W, A S) ----
 * Y = alpha * A V + beta * V + gamma * U, A in CSR with int32 rowptr[n+1],
 * colind[nnz] and values val[nnz] (all device).  V, U, Y are n x w blocks of
 * format dtype (U may be NULL when gamma == 0); val is float64 when dtype is
 * EIG_F64, float32 for EIG_F32 and double-float for EIG_DF64.  Y must not
 * overlap V or U.  The three-term form is one step of the Chebyshev
 * recurrence.  w <= 1024.  Each row is one lane group's work here; inside
 * eig_solve, rows with more than 512 nonzeros (power-law graphs) are split
 * over the warps of a CTA from a list built once at eig_create. */
int eig_spmm(int64_t n, const int32_t *rowptr, const int32_t *colind, const void *val,
             int dtype, int w, const void *V, int64_t ldv, void *Y, int64_t ldy, double alpha,
             double beta, const void *U, int64_t ldu, double gamma, void *stream);

/* ---- a4 / a5 / a8: tall-skinny Gram product (X^T A X, S^T A S, [X,P]^T W)
 * G = U^T V (a x b, float64 row-major with leading dimension ldg, device),
 * U: n x a, V: n x b blocks in the element format that arith implies.
 * sym != 0 declares U^T V symmetric (U == V, or U^T A U with symmetric A):
 * only the upper tile triangle is computed and mirrored.  The reduction over
 * n is split across CTAs into float64 partial tiles held in temporary device
 * memory and summed in a fixed order (deterministic).  a, b <= 4096.
 * arith EIG_ARITH_DF64_TC takes EIG_DF64 blocks and EIG_ARITH_F64_TC EIG_F64
 * blocks (U, V 8-byte aligned, any leading dimension); both also hold the
 * bf16 slices of U and V (12 / 14 bytes per element) in temporary device
 * memory; U == V with equal ldu, ldv and a == b is sliced once. */
int eig_gram(int64_t n, int a, int b, const void *U, int64_t ldu, const void *V, int64_t ldv,
             int arith, int sym, double *G, int64_t ldg, void *stream);

/* ---- device status of the tensor-core products (no counterpart in the
 * paper) ----------------------------------------------------------------
 * The tcgen05 product kernels behind EIG_ARITH_DF64_TC and EIG_ARITH_F64_TC
 * bound every wait on their shared-memory barriers; a wait that runs out
 * ends the kernel early (its results are then wrong) and records the fact on
 * the device.  Returns EIG_ETIMEOUT if that happened since the last call (and
 * clears the record), EIG_ECUDA if the record cannot be read, else EIG_OK.
 * Synchronises the current device.  eig_solve() checks it itself. */
int eig_device_status(void);

/* ---- self-test of the bounded waits (no counterpart in the paper) -------
 * Launches one small tensor-core Gram product (arith EIG_ARITH_DF64_TC or
 * EIG_ARITH_F64_TC, zero operands in temporary device memory) whose copy
 * producer withholds the operands of its first pipeline stage, so that the
 * MMA issuer's wait for them runs out after wait_s seconds (0 < wait_s <= 10);
 * the kernel then frees its resources and ends, and the next
 * eig_device_status() returns EIG_ETIMEOUT.  Synchronises the stream.  It
 * faults nothing and leaves the context usable; the product's result is
 * discarded. */
int eig_tc_wait_selftest(int arith, double wait_s, void *stream);

/* ---- allocation-free Gram product (no counterpart in the paper) ---------
 * The product of eig_gram for the CUDA-core arithmetics (EIG_ARITH_F64,
 * _DF64, _F32, _C32; the tensor-core arithmetics, which need slice buffers,
 * are rejected with EIG_EINVAL), same arguments and result, for callers that
 * cannot allocate device memory while they run: a serving process that gave
 * all of HBM to its own memory pool at start-up, or host code running where a
 * cudaMalloc / cudaFree (which can synchronise the device or fail under
 * memory pressure) is not allowed.  Instead of cudaMallocAsync it uses one
 * fixed scratch array of EIG_NOALLOC_SCRATCH_DOUBLES float64 elements
 * (16 MiB) built into the library; every GPU that loads the library keeps it
 * until the process exits.  Calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *  - Returns EIG_EINVAL when a * b > EIG_NOALLOC_SCRATCH_DOUBLES (the result
 *    would not fit even without splitting the reduction); large n is fine, the
 *    reduction is then split over fewer CTAs.
 *  - The first call on each device looks up the scratch address on that
 *    device (cudaGetSymbolAddress); make that first call before any CUDA
 *    stream capture.
 *  - All calls share the scratch: calls whose kernels may overlap on the GPU
 *    (unordered streams, several host threads) race and must be serialised
 *    by the caller.  Nothing in the scratch needs to start at zero. */
#define EIG_NOALLOC_SCRATCH_DOUBLES (2 * 1024 * 1024)
int eig_gram_noalloc(int64_t n, int a, int b, const void *U, int64_t ldu, const void *V,
                     int64_t ldv, int arith, int sym, double *G, int64_t ldg, void *stream);

/* ---- a4 / a11: block update (X <- S C_X, P <- S C_P, W <- W - Q C) ------
 * Y = U C + beta * Y.  U: n x s block, C: s x c float64 row-major (device,
 * leading dimension ldc), Y: n x c block; U and Y use the element format of
 * arith (EIG_DF64 blocks for EIG_ARITH_DF64_TC, EIG_F64 blocks for
 * EIG_ARITH_F64_TC; both also hold the bf16 slices of U and C, 12 / 14 bytes
 * per element, in temporary device memory).  Y must not overlap U. */
int eig_block_update(int64_t n, int s, int c, const void *U, int64_t ldu, const double *C,
                     int64_t ldc, void *Y, int64_t ldy, double beta, int arith, void *stream);

/* ---- a1 / a2: residual, norms and preconditioning (Eq. conv / rk) -------
 * R = T (AX - X diag(lam)) for the w columns, T = diag(tdiag) (tdiag NULL:
 * identity).  X, AX, R: n x w blocks of format dtype; lam: float64[w]
 * (device); tdiag: n values of format dtype (device) or NULL.  Writes
 * xnorm2[j] = ||x_j||^2 and rnorm2[j] = ||AX_j - lam_j X_j||^2 (before T),
 * float64 device arrays of length w.  R may be NULL (norms only). */
int eig_residual(int64_t n, int w, const void *X, int64_t ldx, const void *AX, int64_t ldax,
                 const double *lam, const void *tdiag, void *R, int64_t ldr, double *xnorm2,
                 double *rnorm2, int dtype, void *stream);

/* ---- a5: CholeskyQR2 in place ("orthogonalize", Algorithms 1-3) --------
 * W (n x w, format of arith) <- W R^{-1} twice, R from the float64 Cholesky
 * factor of the Gram matrix; on breakdown the shifted form of Fukaya et al.
 * (2020) and a third pass.  *status_out (host, may be NULL) receives 0 (plain),
 * 1 (shift used) after the stream is synchronised.  w <= 1024. */
int eig_cholqr2(int64_t n, int w, void *W, int64_t ldw, int arith, int *status_out,
                void *stream);

/* ---- a9: small dense symmetric eigensolver (Rayleigh-Ritz, Algorithms 1-3)
 * A (s x s float64, device, symmetric, leading dimension lda) = Z diag(lam) Z^T
 * with lam ascending.  lam: float64[s], Z: s x s float64 row-major (columns are
 * eigenvectors), both device.  Float64 throughout: Householder
 * tridiagonalisation, eigenvalues by bisection on Sturm counts, eigenvectors
 * by inverse iteration with Gram-Schmidt inside clusters of nearly equal
 * eigenvalues, back-transformation -- the eigensolver of the float64 form
 * (the double-float and mixed forms refine a float32 decomposition instead).
 * A is not modified.  Returns EIG_EBREAKDOWN if the decomposition reported a
 * failure.  s <= 4096. */
int eig_syev(int s, const double *A, int64_t lda, double *lam, double *Z, int64_t ldz,
             void *stream);

/* ---- a10: improved Hetmaniuk-Lehoucq basis selection (Algorithm 3) -----
 * Given all s eigenvectors Z (s x s, ascending), C_P = Z(:, nnow:s) Q with Q the
 * orthonormal QR factor of Z(nlock:nnow, nnow:s)^T, computed by shifted
 * CholeskyQR3 (Fukaya et al. 2020; for a full-rank block the Householder
 * factor up to column signs); CP is s x (nnow - nlock) float64 row-major
 * (device).  Requires s - nnow >= nnow - nlock. */
int eig_hl_trick(int s, int nnow, int nlock, const double *Z, int64_t ldz, double *CP,
                 int64_t ldcp, void *stream);

/* ---- whole solves: eig_create / eig_solve / eig_query ------------------ */
typedef struct {
  int64_t n, nnz;
  const int32_t *rowptr;  /* n + 1 */
  const int32_t *colind;  /* nnz   */
  const void *val;        /* nnz values, float64 or float32 (val_dtype)   */
  int on_device;          /* 1: the three arrays are device pointers (rowptr
                             and colind borrowed, must outlive the handle;
                             values copied); 0: host (copied)              */
  int val_dtype;          /* EIG_F64 (0) or EIG_F32 (1): float32 values are
                             widened to float64 once, at eig_create        */
} eig_csr;

#define EIG_NONE 0     /* fixed block width                                  */
#define EIG_FIX 1      /* Algorithm 6                                         */
#define EIG_SLOPE 2    /* Algorithm 7 with Eq. ckslope                        */
#define EIG_SLOPEK 3   /* Algorithm 7 with Eq. ckslopek                       */

#define EIG_LOBPCG 0   /* Algorithm 3                                         */
#define EIG_CHEB_SI 1  /* Algorithm 1, Chebyshev filter for the solve         */
#define EIG_SD 2       /* Algorithm 2 (steepest descent, no locking)          */

/* Forms of a solve.  In every form the Cholesky factors, the projected
 * eigenproblems and the final residual test run in float64, and the solve
 * ends with a float64 Rayleigh-Ritz pass on the nev converged vectors.
 *  EIG_FORM_F64:   float64 blocks; float64 SpMM and residuals; Gram products
 *                  and block updates on the tensor cores (EIG_ARITH_F64_TC,
 *                  gram_tc = 1) or on the float64 CUDA cores (gram_tc = 0);
 *                  the float64 eigensolver of eig_syev.
 *  EIG_FORM_DF64:  double-float blocks (about 48 significant bits); SpMM and
 *                  residuals on the FP32 pipes; Gram and update on the tensor
 *                  cores (EIG_ARITH_DF64_TC) or the FP32 pipes (gram_tc = 0);
 *                  a float32 eigendecomposition refined in double-float.
 *  EIG_FORM_MIXED: float32 blocks (compensated Gram) until r <= mixed_switch,
 *                  then the double-float form. */
#define EIG_FORM_DF64 0
#define EIG_FORM_F64 1
#define EIG_FORM_MIXED 2

typedef struct {
  int algo;            /* EIG_LOBPCG                                          */
  int form;            /* EIG_FORM_F64                                        */
  double tol;          /* 1e-10: stop when r^(j) <= tol (Eq. rk)              */
  int max_iter;        /* 1000                                                */
  int nes;             /* nev + 5; 0 = default                                */
  int je, js, jp;      /* 12, 2, 10                                           */
  int j_warm;          /* 5                                                   */
  double mu;           /* 1.1                                                 */
  double r_warm;       /* 1e-4                                                */
  int cheb_degree;     /* 12                                                  */
  double cheb_upper;   /* upper bound of the spectrum (0 = normA)             */
  int precond;         /* 0 none, 1 Jacobi T = diag(A)^{-1}                   */
  int deflate_ones;    /* 1: keep every block orthogonal to 1/sqrt(n)         */
  double normA;        /* ||A||_2 used by Eq. conv; 0 (default): eig_create
                          takes the Gershgorin bound of eig_norm_bound, an
                          upper bound (the test is then at most that much
                          stricter)                                          */
  double mixed_switch; /* 1e-5: residual at which MIXED promotes to DF64      */
  const double *X0;    /* n x k_max float64 row-major initial block (required)*/
  int x0_on_device;    /* 1: X0 is a device pointer                           */
  void *stream;        /* cudaStream_t the solve runs on                      */
  int profile;         /* 1: time every kernel class with CUDA events          */
  int expand_powered;  /* EIG_CHEB_SI: 1 = "Powered X_drop" (Sec. 6.4): apply
                          the filter to the saved columns every iteration     */
  int gram_tc;         /* 1 (default): Gram products and block updates of the
                          float64 and double-float blocks on the tensor cores
                          (EIG_ARITH_F64_TC / EIG_ARITH_DF64_TC; slice buffers
                          of 14 / 12 bytes per element for two
                          n x (3 k_max + 1) and two n x (2 k_max + 1)
                          operands, see eig_footprint); 0: on the CUDA cores
                          (float64 FMA / FP32-pipe double-float)             */
  int warm_first;      /* 0 (default): the warm-up gate (end of Sec. 3.2)
                          compares r^(j), the largest Eq. conv residual of the
                          first nev pairs, with r_warm; 1: it compares the
                          residual of the first pair instead (the more
                          aggressive warm-up of the paper's closing remarks,
                          there with r_warm = 1e-1)                          */
  int expand_random;   /* 0 (default): an expansion appends the columns saved
                          at the last shrink (X_drop / S_drop); 1: the
                          'Random' variant of Sec. 6.4 -- it appends as many
                          fresh standard-normal columns instead, entry (i, j)
                          of the e-th expansion's block drawn by
                          Philox4x32-10 (counter (i mod 2^32, i / 2^32,
                          j / 2, e), key = seed) and Box-Muller (cos for even
                          j, sin for odd j) from the float64 uniforms
                          (w0 2^21 + w1 / 2^11 + 1/2) 2^-53 and
                          (w2 2^21 + w3 / 2^11) 2^-53 of its four words    */
  uint64_t seed;       /* key of the 'Random' draws                          */
  int tc_chunk_rows;   /* 0 (default): the slice buffers of the tensor-core
                          products hold all n rows; > 0, a multiple of 128:
                          they hold this many rows and every Gram product and
                          block update runs over row chunks of that size (the
                          Gram's chunks summed in order), so that matrices
                          whose full slice buffers would not fit in HBM (the
                          4M-row graph with k_max = 400) keep the tensor-core
                          products; the slices of [X, P] are then not cached
                          across an orthogonalisation                        */
} eig_options;

/* kernel classes of the per-class statistics (eig_result.kstats) */
#define EIG_K_SPMM 0
#define EIG_K_GRAM 1
#define EIG_K_UPDATE 2
#define EIG_K_RESIDUAL 3
#define EIG_K_CHOL 4
#define EIG_K_SYEV 5
#define EIG_K_HL 6
#define EIG_K_OTHER 7
#define EIG_NKCLASS 8

typedef struct {
  int status;          /* EIG_OK or EIG_ENOTCONV / error of the last solve    */
  int iters;           /* iterations j performed                               */
  int n_shrink, n_expand;
  int nev;
  const double *lambda;   /* host, nev ascending (owned by the handle)        */
  const double *resid;    /* host, nev: ||A v - lambda v|| / normA (float64)  */
  const double *V;        /* device, n x nev float64 row-major (owned)        */
  const double *history;  /* host, r^(j) for j = 1..iters                     */
  const int *widths;      /* host, active width nnow at each iteration        */
  double time_ms;         /* wall time of eig_solve                            */
  double normA;
  /* host, EIG_NKCLASS x 4 (launches, device ms, algorithmic flops,
   * algorithmic DRAM bytes) per kernel class; all zero unless opt.profile.
   * Flops count 2 per multiply-add in the arithmetic of the form; bytes
   * count each n-sized operand read once and each result written once. */
  const double *kstats;
  int64_t launches;      /* kernels this library launched during the solve     */
} eig_result;

typedef struct eig_handle eig_handle;

/* Fill *opt with the defaults listed above (X0 NULL, normA 0). */

/* Gershgorin bound max_i sum_j |a_ij| >= ||A||_2 of a symmetric CSR matrix
 * (host arrays only: A->on_device must be 0), into *out.  eig_create and
 * eig_submit use it when opt->normA is 0.  EIG_EINVAL for a device CSR or a
 * malformed one (n <= 0, rowptr not starting at 0 or not ascending). */
int eig_norm_bound(const eig_csr *A, double *out);
int eig_options_default(eig_options *opt);

/* Validate and allocate a solver for the nev smallest eigenpairs with
 * initial/expanded width k_max (nex).  Requires 1 <= nev <= nes < k_max <= n,
 * opt->X0 != NULL and opt->normA >= 0 (0: the Gershgorin bound, read from
 * the host CSR or, for a device CSR, from one copy of its values).  Device
 * memory: eig_footprint() bytes
 * (for the 128^3 Laplacian with k_max = 128, about 90 GB in the float64 form
 * with the tensor-core products); EIG_ENOMEM if it does not fit. */
int eig_create(const eig_csr *A, int nev, int k_max, int strategy, const eig_options *opt,
               eig_handle **out);
/* Run the solve from X0; blocks until done.  Returns EIG_OK or EIG_ENOTCONV
 * (results of the last iteration are kept) or an error. */
int eig_solve(eig_handle *h);
int eig_query(const eig_handle *h, eig_result *out);
void eig_destroy(eig_handle *h);
const char *eig_strerror(int status);

/* ---- a3: the shrink-and-expand decisions on a scripted history (host
 * only, no device work; no counterpart in the paper) -----------------------
 * Runs the decision rule that eig_solve applies (Algorithms 6 and 7, Eqs.
 * ckslope / ckslopek, the warm-up rule at the end of Sec. 3.2) over the host
 * array r[0 .. m-1] = r^(1) .. r^(m), with the active width nnow starting at
 * nex.  r1 (host, m values, or NULL for r itself) is the residual of the
 * first pair, which the warm-up gate reads when opt->warm_first is set.  For each j it records r^(j), asks whether to expand (nnow = nex when
 * it does), stores width[j-1] = nnow (host array of m ints, or NULL), then
 * asks whether to shrink (nnow = nes when it does) -- the order of the two
 * decision points inside one iteration of eig_solve.  The first max_events
 * events go to events[2 e] = j, events[2 e + 1] = EIG_EVENT_SHRINK or
 * EIG_EVENT_EXPAND (host array of 2 max_events ints, NULL if max_events is
 * 0); *n_events receives the total count.  opt supplies je, js, jp, j_warm,
 * mu, r_warm and warm_first (NULL: the defaults).  Returns EIG_EINVAL for
 * an unknown strategy, nes outside [1, nex), m < 0, a negative or NaN
 * residual, je, js or jp below 1, or a missing array. */
#define EIG_EVENT_SHRINK 1
#define EIG_EVENT_EXPAND 2
int eig_strategy_trace(int strategy, int nes, int nex, const eig_options *opt, const double *r,
                       const double *r1, int m, int *width, int *events, int max_events, int *n_events);

/* ---- serving: many independent solves advanced together ----------------
 * A request loop for the serving workload of many eigenproblems of different
 * n, nev and k_max.  eig_submit copies the request (host CSR, host X0 and the
 * options) into the server and returns a ticket; it rejects (EIG_EREJECT) a
 * request whose device footprint (eig_footprint) exceeds the whole budget.
 * eig_server_step admits queued requests in submission order while their
 * footprint fits mem_budget_bytes and fewer than max_active solves run, then
 * advances every active solve by one iteration (Algorithm 3 / 1 each, with
 * their own shrink / expand decisions); each solve runs on its own CUDA
 * stream so their kernels overlap, and the host part of each iteration runs
 * as soon as that solve's stream has drained (completion order, streams
 * polled).  A solve that finishes inside the step frees its slot and memory
 * at once, and queued requests are admitted into them (their first iteration
 * runs in the same step).  A finished solve's results (eigenvalues,
 * residuals, history, eigenvectors copied to host memory) are kept until
 * eig_release; its device memory and slot are freed at once.  eig_poll sets
 * *ready and fills *out (V is then a HOST pointer, n x nev row-major;
 * time_ms = completion - submission).  Single-threaded: one host thread
 * drives a server. */
typedef struct {
  size_t mem_budget_bytes;   /* device bytes the active solves may hold  */
  int max_active;            /* most solves advanced per step            */
} eig_server_opts;
typedef struct eig_server eig_server;

size_t eig_footprint(int64_t n, int64_t nnz, int nev, int k_max, const eig_options *opt);
int eig_server_create(const eig_server_opts *opts, eig_server **out);
int eig_submit(eig_server *s, const eig_csr *A, int nev, int k_max, int strategy,
               const eig_options *opt, uint64_t *ticket);
int eig_server_step(eig_server *s, int *n_active, int *n_queued);
int eig_poll(eig_server *s, uint64_t ticket, eig_result *out, int *ready);
int eig_release(eig_server *s, uint64_t ticket);
void eig_server_destroy(eig_server *s);

#ifdef __cplusplus
}
#endif
#endif /* EIG_GB300_H */
