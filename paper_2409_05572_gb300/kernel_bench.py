"""Micro-benchmark of single hot-path kernels through the C ABI.

  python -m paper_2409_05572_gb300.kernel_bench --kernel gram --n 2097152 --a 384 --b 384 --sym
  python -m paper_2409_05572_gb300.kernel_bench --kernel update --n 2097152 --a 384 --b 256
  python -m paper_2409_05572_gb300.kernel_bench --kernel spmm --grid 128 --b 128
  python -m paper_2409_05572_gb300.kernel_bench --kernel syev --a 384

Blocks are filled with seeded random double-float data on the device (the
operand values do not change the work of these kernels).  Each kernel is
launched --warmup times, then --reps times between CUDA events on the current
stream; the line printed gives the average time, the algorithmic flops / bytes
of one launch and the rates.  Used for the per-kernel ncu captures.
"""
from __future__ import annotations

import argparse
import json
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", required=True, choices=["gram", "update", "spmm", "syev"])
    ap.add_argument("--n", type=int, default=2097152)
    ap.add_argument("--a", type=int, default=384)
    ap.add_argument("--b", type=int, default=384)
    ap.add_argument("--sym", action="store_true")
    ap.add_argument("--grid", type=int, default=128, help="3D Laplacian grid side for --kernel spmm")
    ap.add_argument("--arith", default="df64", choices=["df64", "df64_tc", "f64", "f32", "c32"],
                    help="df64_tc: double-float blocks, product on the tensor cores (gram, update)")
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)

    import torch

    from . import _lib as L
    from . import workloads as W

    L.load()
    ar = {"df64": L.ARITH_DF64, "df64_tc": L.ARITH_DF64_TC, "f64": L.ARITH_F64, "f32": L.ARITH_F32,
          "c32": L.ARITH_C32}[args.arith]
    if args.arith == "df64_tc" and args.kernel not in ("gram", "update"):
        ap.error("df64_tc applies to --kernel gram and --kernel update")
    g = torch.Generator(device="cuda").manual_seed(1234)

    def block(rows, cols):
        x = torch.randn(rows, cols, generator=g, device="cuda", dtype=torch.float64)
        if args.arith in ("df64", "df64_tc"):
            return L.to_df64(x)
        if args.arith == "f64":
            return x
        return x.float()

    esz = 4 if args.arith in ("f32", "c32") else 8
    n, a, b = args.n, args.a, args.b
    if args.kernel == "gram":
        U = block(n, a)
        V = U if args.sym else block(n, b)
        if args.sym:
            b = a
        G = torch.empty(a, b, dtype=torch.float64, device="cuda")
        fn = lambda: L.eig_gram(n, a, b, U, a, V, b, ar, args.sym, G, b)  # noqa: E731
        flops = n * a * (b + 1) if args.sym else 2.0 * n * a * b
        nbytes = esz * n * (a if args.sym else a + b)
    elif args.kernel == "update":
        U = block(n, a)
        C = torch.randn(a, b, generator=g, device="cuda", dtype=torch.float64)
        Y = block(n, b)
        fn = lambda: L.eig_block_update(n, a, b, U, a, C, b, Y, b, 0.0, ar)  # noqa: E731
        flops = 2.0 * n * a * b
        nbytes = esz * n * (a + b)
    elif args.kernel == "spmm":
        A = W.laplacian_3d(args.grid)
        n = A.n
        rp = torch.as_tensor(A.indptr, device="cuda")
        ci = torch.as_tensor(A.indices, device="cuda")
        vals = torch.as_tensor(A.data, device="cuda")
        dt = {"df64": L.EIG_DF64, "f64": L.EIG_F64, "f32": L.EIG_F32, "c32": L.EIG_F32}[args.arith]
        if dt == L.EIG_DF64:
            vals = L.to_df64(vals)
        elif dt == L.EIG_F32:
            vals = vals.float()
        V = block(n, b)
        Y = torch.empty_like(V)
        fn = lambda: L.eig_spmm(n, rp, ci, vals, dt, b, V, b, Y, b)  # noqa: E731
        flops = 2.0 * A.nnz * b
        nbytes = (4 + esz) * A.nnz + 4 * (n + 1) + 2 * esz * n * b
    else:
        s = a
        M = torch.randn(s, s, generator=g, device="cuda", dtype=torch.float64)
        M = M + M.T
        lam = torch.empty(s, dtype=torch.float64, device="cuda")
        Z = torch.empty(s, s, dtype=torch.float64, device="cuda")
        fn = lambda: L.eig_syev(s, M, s, lam, Z, s)  # noqa: E731
        flops = (4.0 / 3.0 + 6.0) * s ** 3
        nbytes = 0
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    out = {"kernel": args.kernel, "arith": args.arith, "n": n, "a": a, "b": b, "sym": args.sym, "ms": ms,
           "flops": flops, "bytes": nbytes, "tflops": flops / ms / 1e9,
           "gbs": nbytes / ms / 1e6 if nbytes else None}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
