"""ctypes binding of ``libeig_gb300.so`` (C ABI in include/eig_gb300.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Device arrays are passed as torch CUDA tensors (their ``data_ptr``); the
double-float (DF64) element format is carried as float32 tensors whose last
dimension holds the {hi, lo} pair.  There is no CPU fallback: a missing or
unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeig_gb300.so")

# status codes / formats (eig_gb300.h)
EIG_OK, EIG_EINVAL, EIG_ENOMEM, EIG_ENOTCONV, EIG_EBREAKDOWN, EIG_ECUDA, EIG_ETIMEOUT = range(7)
EIG_F64, EIG_F32, EIG_DF64 = 0, 1, 2
ARITH_F64, ARITH_DF64, ARITH_F32, ARITH_C32 = 0, 1, 2, 3
ARITH_DF64_TC = 4  # eig_gram / eig_block_update: double-float blocks, tensor-core product
ARITH_F64_TC = 5   # eig_gram / eig_block_update: float64 blocks, tensor-core product
STRATEGIES = {"none": 0, "fix": 1, "slope": 2, "slopek": 3}
ALGOS = {"lobpcg": 0, "chebsi": 1, "sd": 2}
FORMS = {"df64": 0, "f64": 1, "mixed": 2}

EXPORTS = ("eig_convert", "eig_spmm", "eig_gram", "eig_gram_noalloc", "eig_block_update", "eig_residual",
           "eig_cholqr2", "eig_syev", "eig_hl_trick", "eig_options_default", "eig_create", "eig_solve",
           "eig_query", "eig_destroy", "eig_strerror", "eig_footprint", "eig_server_create", "eig_submit",
           "eig_server_step", "eig_poll", "eig_release", "eig_server_destroy", "eig_device_status",
           "eig_strategy_trace", "eig_tc_wait_selftest", "eig_norm_bound")


class EigError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {msg} (status {code})")
        self.code = code


class eig_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int), ("val_dtype", C.c_int)]


class eig_options(C.Structure):
    _fields_ = [("algo", C.c_int), ("form", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("nes", C.c_int), ("je", C.c_int), ("js", C.c_int), ("jp", C.c_int), ("j_warm", C.c_int),
                ("mu", C.c_double), ("r_warm", C.c_double), ("cheb_degree", C.c_int),
                ("cheb_upper", C.c_double), ("precond", C.c_int), ("deflate_ones", C.c_int),
                ("normA", C.c_double), ("mixed_switch", C.c_double), ("X0", C.c_void_p),
                ("x0_on_device", C.c_int), ("stream", C.c_void_p), ("profile", C.c_int),
                ("expand_powered", C.c_int), ("gram_tc", C.c_int), ("warm_first", C.c_int),
                ("expand_random", C.c_int), ("seed", C.c_uint64), ("tc_chunk_rows", C.c_int)]


class eig_server_opts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_active", C.c_int)]


class eig_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("n_shrink", C.c_int), ("n_expand", C.c_int),
                ("nev", C.c_int), ("lambda_", C.POINTER(C.c_double)), ("resid", C.POINTER(C.c_double)),
                ("V", C.c_void_p), ("history", C.POINTER(C.c_double)), ("widths", C.POINTER(C.c_int)),
                ("time_ms", C.c_double), ("normA", C.c_double), ("kstats", C.POINTER(C.c_double)),
                ("launches", C.c_int64)]

KCLASSES = ("spmm", "gram", "update", "residual", "chol", "syev", "hl", "other")


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    p, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "eig_convert": [i64, p, i32, p, i32, p],
        "eig_spmm": [i64, p, p, p, i32, i32, p, i64, p, i64, d, d, p, i64, d, p],
        "eig_gram": [i64, i32, i32, p, i64, p, i64, i32, i32, p, i64, p],
        "eig_gram_noalloc": [i64, i32, i32, p, i64, p, i64, i32, i32, p, i64, p],
        "eig_device_status": [],
        "eig_tc_wait_selftest": [i32, d, p],
        "eig_block_update": [i64, i32, i32, p, i64, p, i64, p, i64, d, i32, p],
        "eig_residual": [i64, i32, p, i64, p, i64, p, p, p, i64, p, p, i32, p],
        "eig_cholqr2": [i64, i32, p, i64, i32, C.POINTER(C.c_int), p],
        "eig_syev": [i32, p, i64, p, p, i64, p],
        "eig_hl_trick": [i32, i32, i32, p, i64, p, i64, p],
        "eig_options_default": [C.POINTER(eig_options)],
        "eig_create": [C.POINTER(eig_csr), i32, i32, i32, C.POINTER(eig_options), C.POINTER(C.c_void_p)],
        "eig_solve": [p],
        "eig_query": [p, C.POINTER(eig_result)],
        "eig_destroy": [p],
        "eig_strerror": [i32],
        "eig_server_create": [C.POINTER(eig_server_opts), C.POINTER(C.c_void_p)],
        "eig_submit": [p, C.POINTER(eig_csr), i32, i32, i32, C.POINTER(eig_options), C.POINTER(C.c_uint64)],
        "eig_server_step": [p, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "eig_poll": [p, C.c_uint64, C.POINTER(eig_result), C.POINTER(C.c_int)],
        "eig_release": [p, C.c_uint64],
        "eig_server_destroy": [p],
        "eig_footprint": [i64, i64, i32, i32, C.POINTER(eig_options)],
        "eig_strategy_trace": [i32, i32, i32, C.POINTER(eig_options), p, p, i32, p, p, i32, C.POINTER(C.c_int)],
        "eig_norm_bound": [C.POINTER(eig_csr), C.POINTER(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.eig_destroy.restype = None
    lib.eig_server_destroy.restype = None
    lib.eig_footprint.restype = C.c_size_t
    lib.eig_strerror.restype = C.c_char_p
    _lib = lib
    return lib


def _check(fn, code):
    if code != EIG_OK:
        raise EigError(fn, code, load().eig_strerror(code).decode())
    return code


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _fmt(t, dtype_code=None):
    """Element format of a tensor: float64 -> F64, float32 with trailing
    pair dimension -> DF64 when requested, float32 -> F32."""
    import torch
    if dtype_code is not None:
        return dtype_code
    if t.dtype == torch.float64:
        return EIG_F64
    if t.dtype == torch.float32:
        return EIG_F32
    raise TypeError(t.dtype)


# ---------------------------------------------------------------------------
# format helpers
# ---------------------------------------------------------------------------
def to_df64(x, stream=None):
    """float64 CUDA tensor -> double-float tensor (..., 2) float32."""
    import torch
    x = x.contiguous()
    out = torch.empty(*x.shape, 2, dtype=torch.float32, device=x.device)
    _check("eig_convert", load().eig_convert(x.numel(), _ptr(x), EIG_F64, _ptr(out), EIG_DF64, _stream(stream)))
    return out


def from_df64(x, stream=None):
    import torch
    x = x.contiguous()
    out = torch.empty(*x.shape[:-1], dtype=torch.float64, device=x.device)
    _check("eig_convert", load().eig_convert(out.numel(), _ptr(x), EIG_DF64, _ptr(out), EIG_F64, _stream(stream)))
    return out


def convert(src, src_dtype, dst, dst_dtype, count, stream=None):
    return _check("eig_convert", load().eig_convert(count, _ptr(src), src_dtype, _ptr(dst), dst_dtype,
                                                    _stream(stream)))


# ---------------------------------------------------------------------------
# step-level entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def eig_spmm(n, rowptr, colind, val, dtype, w, V, ldv, Y, ldy, alpha=1.0, beta=0.0, U=None, ldu=0,
             gamma=0.0, stream=None):
    return _check("eig_spmm", load().eig_spmm(n, _ptr(rowptr), _ptr(colind), _ptr(val), dtype, w, _ptr(V), ldv,
                                              _ptr(Y), ldy, alpha, beta, _ptr(U), ldu, gamma, _stream(stream)))


def eig_gram(n, a, b, U, ldu, V, ldv, arith, sym, G, ldg, stream=None):
    return _check("eig_gram", load().eig_gram(n, a, b, _ptr(U), ldu, _ptr(V), ldv, arith, int(sym), _ptr(G), ldg,
                                              _stream(stream)))


EVENT_SHRINK, EVENT_EXPAND = 1, 2


def eig_strategy_trace(strategy, nes, nex, r, r1=None, **opts):
    """The shrink-and-expand decisions eig_solve takes on the scripted
    residual history r^(1) .. r^(m) (host only, no device work); r1, if
    given, is the first pair's residual history (read by the warm-up gate
    when warm_first is set).  Returns (events, widths): events as
    (j, "shrink" | "expand") in order, widths[j-1] the active width of
    iteration j.  opts: je, js, jp, j_warm, mu, r_warm, warm_first."""
    import numpy as np
    lib = load()
    rr = np.ascontiguousarray(r, dtype=np.float64)
    m = int(rr.size)
    r1a = None if r1 is None else np.ascontiguousarray(r1, dtype=np.float64)
    if r1a is not None and r1a.size != m:
        raise ValueError("r1 must have the length of r")
    width = np.zeros(max(m, 1), dtype=np.int32)
    cap = 2 * m + 2
    ev = np.zeros(2 * cap, dtype=np.int32)
    n_ev = C.c_int(0)
    opt = None
    if opts:
        o = eig_options()
        lib.eig_options_default(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        opt = C.byref(o)
    _check("eig_strategy_trace", lib.eig_strategy_trace(STRATEGIES[strategy], nes, nex, opt,
                                                        rr.ctypes.data if m else None,
                                                        r1a.ctypes.data if (r1a is not None and m) else None, m,
                                                        width.ctypes.data, ev.ctypes.data, cap, C.byref(n_ev)))
    names = {EVENT_SHRINK: "shrink", EVENT_EXPAND: "expand"}
    events = [(int(ev[2 * e]), names[int(ev[2 * e + 1])]) for e in range(min(n_ev.value, cap))]
    return events, [int(x) for x in width[:m]]


def device_status():
    """EIG_ETIMEOUT if a bounded wait inside a tensor-core product ran out
    since the last call (clears it), else 0; synchronises the device."""
    return int(load().eig_device_status())


def eig_tc_wait_selftest(arith, wait_s, stream=None):
    """Launch a tensor-core Gram product whose first stage is withheld, so a
    bounded wait runs out after wait_s seconds; device_status() then reports
    EIG_ETIMEOUT."""
    return _check("eig_tc_wait_selftest", load().eig_tc_wait_selftest(arith, wait_s, _stream(stream)))


def eig_gram_noalloc(n, a, b, U, ldu, V, ldv, arith, sym, G, ldg, stream=None):
    """eig_gram without device allocation (fixed built-in scratch, shared by
    all calls; a * b must not exceed NOALLOC_SCRATCH_DOUBLES)."""
    return _check("eig_gram_noalloc", load().eig_gram_noalloc(n, a, b, _ptr(U), ldu, _ptr(V), ldv, arith, int(sym),
                                                              _ptr(G), ldg, _stream(stream)))


NOALLOC_SCRATCH_DOUBLES = 2 * 1024 * 1024


def eig_block_update(n, s, c, U, ldu, Cm, ldc, Y, ldy, beta, arith, stream=None):
    return _check("eig_block_update", load().eig_block_update(n, s, c, _ptr(U), ldu, _ptr(Cm), ldc, _ptr(Y), ldy,
                                                              beta, arith, _stream(stream)))


def eig_residual(n, w, X, ldx, AX, ldax, lam, tdiag, R, ldr, xnorm2, rnorm2, dtype, stream=None):
    return _check("eig_residual", load().eig_residual(n, w, _ptr(X), ldx, _ptr(AX), ldax, _ptr(lam), _ptr(tdiag),
                                                      _ptr(R), ldr, _ptr(xnorm2), _ptr(rnorm2), dtype,
                                                      _stream(stream)))


def eig_cholqr2(n, w, W, ldw, arith, stream=None):
    st = C.c_int(0)
    _check("eig_cholqr2", load().eig_cholqr2(n, w, _ptr(W), ldw, arith, C.byref(st), _stream(stream)))
    return st.value


def eig_syev(s, A, lda, lam, Z, ldz, stream=None):
    return _check("eig_syev", load().eig_syev(s, _ptr(A), lda, _ptr(lam), _ptr(Z), ldz, _stream(stream)))


def eig_hl_trick(s, nnow, nlock, Z, ldz, CP, ldcp, stream=None):
    return _check("eig_hl_trick", load().eig_hl_trick(s, nnow, nlock, _ptr(Z), ldz, _ptr(CP), ldcp,
                                                      _stream(stream)))


# ---------------------------------------------------------------------------
# whole solves: eig_create / eig_solve / eig_query
# ---------------------------------------------------------------------------
class Solver:
    """Owns an eig_handle.  ``A`` is a workloads.CSR (host arrays, copied to
    the device) or a tuple of CUDA tensors (rowptr int32, colind int32,
    val float64) that must outlive the solver."""

    def __init__(self, A, nev, k_max, strategy="fix", X0=None, normA=None, algo="lobpcg", form="f64",
                 tol=1e-10, max_iter=1000, nes=0, stream=None, **kw):
        lib = load()
        self._keep = []
        csr = eig_csr()
        if isinstance(A, tuple):
            rp, ci, va = A
            csr.n, csr.nnz = rp.numel() - 1, ci.numel()
            csr.rowptr, csr.colind, csr.val = rp.data_ptr(), ci.data_ptr(), va.data_ptr()
            csr.on_device = 1
            csr.val_dtype = EIG_F32 if str(va.dtype) == "torch.float32" else EIG_F64
            self._keep += [rp, ci, va]
        else:
            rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
            ci = np.ascontiguousarray(A.indices, dtype=np.int32)
            vdt = np.float32 if np.asarray(A.data).dtype == np.float32 else np.float64
            va = np.ascontiguousarray(A.data, dtype=vdt)
            self._keep += [rp, ci, va]
            csr.n, csr.nnz = A.n, ci.size
            csr.rowptr, csr.colind, csr.val = rp.ctypes.data, ci.ctypes.data, va.ctypes.data
            csr.on_device = 0
            csr.val_dtype = EIG_F32 if vdt == np.float32 else EIG_F64
        opt = eig_options()
        lib.eig_options_default(C.byref(opt))
        opt.algo = ALGOS[algo]
        opt.form = FORMS[form]
        opt.tol = tol
        opt.max_iter = max_iter
        opt.nes = nes
        for k, v in kw.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, v)
        # None: eig_create takes the Gershgorin bound of ||A||_2
        opt.normA = 0.0 if normA is None else float(normA)
        if X0 is None:
            raise ValueError("X0 (n x k_max float64) is required")
        if hasattr(X0, "data_ptr"):
            opt.X0 = X0.data_ptr()
            opt.x0_on_device = 1
            self._keep.append(X0)
        else:
            x0 = np.ascontiguousarray(X0, dtype=np.float64)
            self._keep.append(x0)
            opt.X0 = x0.ctypes.data
            opt.x0_on_device = 0
        opt.stream = _stream(stream).value if stream is not None or _torch_cuda() else None
        self.n, self.nev = csr.n, nev
        h = C.c_void_p()
        _check("eig_create", lib.eig_create(C.byref(csr), nev, k_max, STRATEGIES[strategy], C.byref(opt),
                                            C.byref(h)))
        self._h = h

    def solve(self):
        code = load().eig_solve(self._h)
        if code not in (EIG_OK, EIG_ENOTCONV):
            _check("eig_solve", code)
        return self.query()

    def query(self):
        r = eig_result()
        _check("eig_query", load().eig_query(self._h, C.byref(r)))
        nev, it = r.nev, r.iters
        out = {
            "status": r.status, "iters": it, "n_shrink": r.n_shrink, "n_expand": r.n_expand,
            "lam": np.ctypeslib.as_array(r.lambda_, (nev,)).copy() if r.lambda_ else None,
            "resid": np.ctypeslib.as_array(r.resid, (nev,)).copy() if r.resid else None,
            "history": np.ctypeslib.as_array(r.history, (it,)).copy() if r.history and it else np.zeros(0),
            "widths": (np.ctypeslib.as_array(r.widths, (max(it - (1 if r.status == EIG_OK else 0), 0),)).copy()
                       if r.widths else np.zeros(0, dtype=np.int32)),
            "time_ms": r.time_ms, "V_ptr": r.V, "launches": int(r.launches), "normA": r.normA,
        }
        if r.kstats:
            ks = np.ctypeslib.as_array(r.kstats, (len(KCLASSES), 4)).copy()
            out["kstats"] = {name: {"launches": int(ks[i, 0]), "ms": ks[i, 1], "flops": ks[i, 2],
                                    "bytes": ks[i, 3]} for i, name in enumerate(KCLASSES)}
        return out

    def V(self):
        """n x nev float64 CUDA tensor copy of the eigenvectors."""
        import torch
        r = eig_result()
        _check("eig_query", load().eig_query(self._h, C.byref(r)))
        out = torch.empty(self.n, self.nev, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        _cuda_copy_d2d(out.data_ptr(), r.V, out.numel() * 8)
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().eig_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def _cuda_copy_d2d(dst, src, nbytes):
    """Device-to-device copy through the library's conversion entry point
    (float64 -> float64)."""
    _check("eig_convert", load().eig_convert(nbytes // 8, C.c_void_p(src), EIG_F64, C.c_void_p(dst), EIG_F64,
                                             _stream(None)))


def make_options(algo="lobpcg", form="f64", tol=1e-10, max_iter=1000, nes=0, normA=None, **kw):
    opt = eig_options()
    load().eig_options_default(C.byref(opt))
    opt.algo = ALGOS[algo]
    opt.form = FORMS[form]
    opt.tol = tol
    opt.max_iter = max_iter
    opt.nes = nes
    for k, v in kw.items():
        if not hasattr(opt, k):
            raise TypeError(f"unknown option {k}")
        setattr(opt, k, v)
    if normA is not None:
        opt.normA = float(normA)
    return opt


def norm_bound(A):
    """eig_norm_bound: the Gershgorin bound of ||A||_2 of a host CSR matrix."""
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    vdt = np.float32 if np.asarray(A.data).dtype == np.float32 else np.float64
    va = np.ascontiguousarray(A.data, dtype=vdt)
    csr = eig_csr(A.n, ci.size, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0,
                  EIG_F32 if vdt == np.float32 else EIG_F64)
    out = C.c_double()
    _check("eig_norm_bound", load().eig_norm_bound(C.byref(csr), C.byref(out)))
    return out.value


def footprint(n, nnz, nev, k_max, **opts):
    opt = make_options(**opts)
    return int(load().eig_footprint(n, nnz, nev, k_max, C.byref(opt)))


class Server:
    """Serving loop (eig_server_*): submit host problems, step, poll."""

    def __init__(self, mem_budget_bytes, max_active=64):
        o = eig_server_opts(mem_budget_bytes, max_active)
        h = C.c_void_p()
        _check("eig_server_create", load().eig_server_create(C.byref(o), C.byref(h)))
        self._h = h

    def submit(self, A, X0, nev, k_max, strategy="fix", normA=None, **opts):
        rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        vdt = np.float32 if np.asarray(A.data).dtype == np.float32 else np.float64
        va = np.ascontiguousarray(A.data, dtype=vdt)
        x0 = np.ascontiguousarray(X0, dtype=np.float64)
        csr = eig_csr(A.n, ci.size, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0,
                      EIG_F32 if vdt == np.float32 else EIG_F64)
        opt = make_options(normA=normA, **opts)
        opt.X0 = x0.ctypes.data
        opt.x0_on_device = 0
        t = C.c_uint64()
        _check("eig_submit", load().eig_submit(self._h, C.byref(csr), nev, k_max, STRATEGIES[strategy],
                                               C.byref(opt), C.byref(t)))
        return t.value

    def step(self):
        a, q = C.c_int(), C.c_int()
        _check("eig_server_step", load().eig_server_step(self._h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, ticket, n=None):
        r = eig_result()
        ready = C.c_int()
        _check("eig_poll", load().eig_poll(self._h, ticket, C.byref(r), C.byref(ready)))
        if not ready.value:
            return None
        nev, it = r.nev, r.iters
        out = {"status": r.status, "iters": it, "n_shrink": r.n_shrink, "n_expand": r.n_expand,
               "lam": np.ctypeslib.as_array(r.lambda_, (nev,)).copy() if r.lambda_ else None,
               "resid": np.ctypeslib.as_array(r.resid, (nev,)).copy() if r.resid else None,
               "latency_ms": r.time_ms}
        if r.V and n is not None:
            out["V"] = np.ctypeslib.as_array(C.cast(r.V, C.POINTER(C.c_double)), (n, nev)).copy()
        return out

    def release(self, ticket):
        _check("eig_release", load().eig_release(self._h, ticket))

    def close(self):
        if getattr(self, "_h", None):
            load().eig_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
