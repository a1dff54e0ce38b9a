#!/usr/bin/env python3
"""Benchmark: converged eigenpairs/s at 1e-8 residual of the shrink-and-expand
LOBPCG on one GB300, against the fixed-block solver.

Workload (default): 3D Dirichlet 7-point Laplacian on a 128^3 grid
(n = 2,097,152, nnz = 14,581,760, int32 CSR), the 64 smallest eigenpairs,
LOBPCG with k_max = 128 (nes = 69), Gaussian X0 (Philox seed 1), residual
tolerance 1e-8, strategy `fix`, float64 form: float64 blocks, float64 SpMM,
Gram products and block updates on the tensor cores by an exact seven-slice
splitting (float64-class accuracy), float64 small dense steps.  After the
timed solves the same workload is solved once under each other strategy
(`none` = the fixed block, `slope`, `slopek`), and `fixed_block` /
`strategies` report them.

A step is one whole solve: X0 -> 64 eigenpairs whose relative residual
||A v - lambda v|| / ||A|| is at most 1e-8 (checked in float64 after every
solve).  value = nev / (seconds per solve) summed over ranks.  Inputs are
resident in HBM when the timed region starts; the blocks (4.3 GB each) are
far larger than L2, so no separate L2 flush is needed.

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on the host cores: one step is one iteration of the oracle's own
LOBPCG solve of the same workload (the first W iterations untimed), and the
eigenpairs/s it reports projects the timed mean iteration onto the
iteration count of a whole solve (labelled as a projection).

--kernel times one kernel class on its own (micro-benchmark for ncu).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2409_05572_gb300 import workloads as W  # noqa: E402

METRIC = "converged eigenpairs/s at 1e-8 residual vs fixed-block FP64; p50/p99 latency"
UNIT = "eigenpairs/s"

# DRAM traffic / algorithmic bytes of the tensor-core classes of the float64
# form (slicing + product kernels), from one ncu capture of the current
# kernels at n = 262,144 (`bench.py --kernel gram --n 262144 --a 384 --sym
# --arith f64_tc` and `--kernel update ... --a 384 --b 256`; 384-column
# operands; the Gram class reads U once, 0.805 GB; the update class reads U
# and writes Y, 1.342 GB): column slicer 0.805 GB read + 1.356 GB written,
# Gram product 1.417 + 0.003 GB; row slicer 0.805 + 1.357 GB, update product
# 1.414 + 0.511 GB.  Traffic grows with n.
TC_TRAFFIC_RATIO = {"gram": (0.805 + 1.356 + 1.417 + 0.003) / 0.805,
                    "update": (0.805 + 1.357 + 1.414 + 0.511) / 1.342}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def bf16_sustained():
    """Sustained bf16 tensor rate (TFLOP/s) for kernels timed inside a long
    step: the measured seconds-long cuBLAS loop, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return d["bf16_tflops_sustained"], "measured (sustained cuBLAS bf16 GEMM)"
    return 1700.0, "fallback (sustained)"


# The tensor-core Gram and update cut each operand into exact bf16 slices
# and form the slice products of the kept levels: 28 bf16 multiply-adds per
# float64 multiply-add (seven slices, levels 0..6), 21 per double-float one
# (six slices, levels 0..5).
TC_MMA_PER_MAC = {"f64": 28, "df64": 21}


# FP32 issue rate measured on this machine's GB300 (152 SMs, FFMA, 72.6 TFLOP/s
# = 36.3 T instructions/s); a double-float multiply-add is 11 FP32
# instructions plus a renormalisation every 32, i.e. 11.1 on average.
FP32_INSTR_PER_S = 36.3e12
DF64_INSTR_PER_MAC = 11.1
DF64_PEAK_TFLOPS = 2.0 * FP32_INSTR_PER_S / DF64_INSTR_PER_MAC / 1e12
FP64_PEAK_TFLOPS = 1.01   # measured native FP64 FMA rate


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# options of the expansion variants of Sec. 6.4
EXPAND_OPTS = {"drop": {}, "powered": {"expand_powered": 1}, "random": {"expand_random": 1, "seed": 2024}}


def make_workload(name):
    if name == "c2":
        L = 128
        A = W.laplacian_3d(L)
        return dict(A=A, nev=64, k_max=128, normA=W.dirichlet_norm((L, L, L)), seed=1, tol=1e-8,
                    desc="3D Dirichlet 7-point Laplacian 128^3 (n=2097152, nnz=14581760), nev=64, "
                         "LOBPCG k_max=128 nes=69, Gaussian X0 seed 1, residual 1e-8",
                    exact=dirichlet_lowest((L, L, L), 64))
    if name == "c3":
        A = W.anderson_3d(100, seed=2)
        return dict(A=A, nev=128, k_max=256, normA=W.norm_estimate(A), seed=2, tol=1e-8, algo="chebsi",
                    extra=dict(cheb_degree=12, cheb_upper=W.gershgorin_bound(A)),
                    desc="3D Anderson Hamiltonian 100^3 periodic, disorder U[-8.25,8.25] seed 2 (n=1000000, "
                         "nnz=7000000), nev=128, Chebyshev-filtered subspace iteration degree 12, k_max=256, "
                         "residual 1e-8", exact=None)
    if name == "c4":
        A = W.graph_laplacian(4_000_000, seed=3)
        return dict(A=A, nev=200, k_max=400, normA=W.norm_estimate(A), seed=3, tol=1e-8, algo="lobpcg",
                    extra=dict(precond=1, deflate_ones=1, tc_chunk_rows=1048576),
                    desc=f"graph Laplacian, power-law degrees (exponent 2.5, mean 10), n={A.n}, nnz={A.nnz}, "
                         "nev=200 above the null vector, LOBPCG k_max=400 + Jacobi, residual 1e-8",
                    exact=None)
    if name == "c2s":   # reduced stand-in for quick checks
        L = 48
        A = W.laplacian_3d(L)
        return dict(A=A, nev=64, k_max=128, normA=W.dirichlet_norm((L, L, L)), seed=1, tol=1e-8,
                    desc="3D Dirichlet 7-point Laplacian 48^3, nev=64, LOBPCG k_max=128",
                    exact=dirichlet_lowest((L, L, L), 64))
    raise ValueError(name)


def dirichlet_lowest(dims, k):
    axes = [4 * np.sin(np.arange(1, min(d, k) + 1) * np.pi / (2 * (d + 1))) ** 2 for d in dims]
    tot = axes[0]
    for a in axes[1:]:
        tot = np.add.outer(tot, a).ravel()
    return np.sort(tot)[:k]


def reduce_step_time(ms_step, dist=None, device="cpu"):
    """Max over ranks of the per-rank step time (the job is as slow as its
    slowest replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms_step)
    import torch
    t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nev, world_size, ms_step):
    """Whole-job eigenpairs/s: every rank solves its own replica."""
    return world_size * nev / (ms_step / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_iterations(wl, strategy, iters):
    """Run the FP64 oracle's own LOBPCG solve of the workload for `iters`
    iterations (Algorithm 3 as it stands, on the host cores, BLAS threads =
    affinity cores) and return the wall time of the set-up plus each
    iteration: times[0] = set-up + iteration 1, times[j] = iteration j + 1
    (stamped by the oracle's per-iteration observer after each Rayleigh-Ritz
    step)."""
    from oracle.lobpcg import lobpcg as o_lobpcg
    A, nev, k = wl["A"], wl["nev"], wl["k_max"]
    X0 = W.gaussian_block(A.n, k, wl["seed"])
    stamps = []
    t0 = time.perf_counter()
    o_lobpcg(A, X0, nev, nev + 5, strategy, tol=0.5 * wl["tol"], normA=wl["normA"], max_iter=iters,
             observer=lambda *a: stamps.append(time.perf_counter()))
    prev, out = t0, []
    for t in stamps:
        out.append(t - prev)
        prev = t
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores.  A step
    is one iteration of the oracle's solve of the same workload; the first
    `warmup` iterations (the first includes the set-up) are not timed."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = make_workload(args.workload)
    if wl.get("algo", "lobpcg") != "lobpcg":
        print(json.dumps({"impl": "reference", "unavailable": "the timed oracle arm covers the LOBPCG workloads"}))
        return 0
    nev = wl["nev"]
    cores = len(os.sched_getaffinity(0))
    t_all = time.perf_counter()
    times = oracle_iterations(wl, args.strategy, args.warmup + args.steps)
    timed = times[args.warmup:]
    ms_iter = 1e3 * statistics.mean(timed)
    sec_solve = ms_iter / 1e3 * args.ref_iters
    value = nev / sec_solve
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_iter, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["desc"], "strategy": args.strategy,
                       "step": "one iteration of the oracle's LOBPCG solve (iterations "
                               f"{args.warmup + 1}..{args.warmup + args.steps} timed)"},
            "projection": {"iterations_per_solve": args.ref_iters,
                           "source": "iteration count of the GPU solve of the same workload",
                           "seconds_per_solve": sec_solve,
                           "note": "value = nev / (timed mean iteration x iterations_per_solve); the early "
                                   "iterations run at the full width k_max, later ones are narrower after "
                                   "shrinks and locking, so this overstates the solve time somewhat"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed iterations of the oracle's own solve "
                                       f"(mean {ms_iter / 1e3:.2f} s), projected to {args.ref_iters} iterations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(wl, strategy, iters):
    """The oracle as it stands on a bounded sample: the set-up and first
    iteration of its own solve of the workload, projected to the GPU
    solve's iteration count."""
    cores = len(os.sched_getaffinity(0))
    t = oracle_iterations(wl, strategy, 1)[0]
    sec = t * iters
    return {"value": wl["nev"] / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"set-up + first iteration of the FP64 oracle's LOBPCG solve of this workload "
                      f"({t:.2f} s, BLAS threads = affinity cores), projected to the GPU solve's {iters} "
                      "iterations"}


def run_serving(args):
    """c5: open-loop replay of the Poisson request stream (seed 4) through the
    serving loop (mixed form by default, strategy fix, residual 1e-8).
    Requests are submitted when their arrival time has passed; value = sum of
    nev / makespan (first arrival to last completion); latency = completion -
    arrival.  Unless --no-compare, the same requests are then solved one at a
    time in the plain float64 form (eig_solve per request, in arrival order)
    and reported beside it as `one_at_a_time_f64`."""
    import torch
    from paper_2409_05572_gb300 import _lib as L
    torch.cuda.set_device(0)
    L.load()
    reqs = W.serving_stream(count=args.requests, rate=200.0, seed=4)
    prepared = []
    for r in reqs:
        A = r.matrix()
        normA = W.dirichlet_norm(r.dims) + float(r.diag_shift.max())
        prepared.append((r, A, normA, W.gaussian_block(A.n, r.k_max, r.seed)))
    opts = dict(form=args.form, tol=0.5e-8, max_iter=args.max_iter)
    srv = L.Server(int(args.budget_gb * 2**30), args.max_active)
    clocks = Clocks(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending = list(range(len(prepared)))
    live = {}
    done = {}
    while pending or live:
        now = time.perf_counter() - t0
        while pending and prepared[pending[0]][0].arrival_s <= now:
            i = pending.pop(0)
            r, A, normA, X0 = prepared[i]
            live[srv.submit(A, X0, r.nev, r.k_max, "fix", normA=normA, **opts)] = i
        if not live:
            time.sleep(max(0.0, prepared[pending[0]][0].arrival_s - now))
            continue
        srv.step()
        for t in list(live):
            got = srv.poll(t)
            if got is not None:
                i = live.pop(t)
                done[i] = (got, time.perf_counter() - t0)
                srv.release(t)
    makespan = max(tc for _, tc in done.values()) - prepared[0][0].arrival_s
    clk = clocks.stop()
    lat = np.array([(tc - prepared[i][0].arrival_s) * 1e3 for i, (_, tc) in done.items()])
    pairs = sum(prepared[i][0].nev for i in done)
    ok = all(g["status"] == 0 and float(np.max(g["resid"])) <= 1e-8 for g, _ in done.values())
    line = {"metric": METRIC, "value": pairs / makespan, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": makespan * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed(f32->df64)" if args.form == "mixed" else args.form, "data": "synthetic",
            "config": {"workload": f"serving stream: first {len(prepared)} of the Poisson(200/s) stream, seed 4; "
                                   "2D/3D Dirichlet Laplacian + U[0,1] diagonal, n log-uniform [1e4,1e6], "
                                   f"nev U{{8..128}}, k_max=2 nev; {args.form} LOBPCG + fix, residual 1e-8",
                       "budget_gb": args.budget_gb, "max_active": args.max_active},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "all_converged": bool(ok), "requests": len(done), "eigenpairs": int(pairs), "clocks": clk}
    srv.close()
    if not args.no_compare:
        # the same requests one at a time, plain float64, each solve on its own
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        per = []
        for r, A, normA, X0 in prepared:
            ts = time.perf_counter()
            s = L.Solver(A, nev=r.nev, k_max=r.k_max, strategy="fix", X0=X0, normA=normA, form="f64",
                         tol=0.5e-8, max_iter=args.max_iter)
            o = s.solve()
            s.close()
            per.append((time.perf_counter() - ts, o["status"]))
        tot = time.perf_counter() - t1
        line["one_at_a_time_f64"] = {"value": pairs / tot, "unit": UNIT, "seconds": tot,
                                     "all_converged": all(st == 0 for _, st in per),
                                     "serving_speedup": (pairs / makespan) / (pairs / tot)}
    print(json.dumps(line), flush=True)
    return 0


def run_kernel(args):
    """--kernel: one hot-path kernel class through the C ABI on seeded random
    device blocks (the operand values do not change the work), --warmup
    launches then --steps launches between CUDA events on the current
    stream; prints the average time and the algorithmic flops / bytes of
    one call.  Used for the per-kernel ncu captures."""
    import torch
    from paper_2409_05572_gb300 import _lib as L
    torch.cuda.set_device(0)
    L.load()
    ar = {"df64": L.ARITH_DF64, "df64_tc": L.ARITH_DF64_TC, "f64": L.ARITH_F64, "f64_tc": L.ARITH_F64_TC,
          "f32": L.ARITH_F32, "c32": L.ARITH_C32}[args.arith]
    g = torch.Generator(device="cuda").manual_seed(1234)

    def block(rows, cols):
        x = torch.randn(rows, cols, generator=g, device="cuda", dtype=torch.float64)
        if args.arith in ("df64", "df64_tc"):
            return L.to_df64(x)
        if args.arith in ("f64", "f64_tc"):
            return x
        return x.float()

    esz = 4 if args.arith in ("f32", "c32") else 8
    n, a, b = args.n, args.a, args.b
    if args.kernel == "gram":
        U = block(n, a)
        V = U if args.sym else block(n, b)
        b = a if args.sym else b
        G = torch.empty(a, b, dtype=torch.float64, device="cuda")
        fn = lambda: L.eig_gram(n, a, b, U, a, V, b, ar, args.sym, G, b)  # noqa: E731
        flops = n * a * (b + 1.0) if args.sym else 2.0 * n * a * b
        nbytes = esz * n * (a if args.sym else a + b)
    elif args.kernel == "update":
        U = block(n, a)
        Cm = torch.randn(a, b, generator=g, device="cuda", dtype=torch.float64)
        Y = block(n, b)
        fn = lambda: L.eig_block_update(n, a, b, U, a, Cm, b, Y, b, 0.0, ar)  # noqa: E731
        flops = 2.0 * n * a * b
        nbytes = esz * n * (a + b)
    elif args.kernel == "spmm":
        A = W.laplacian_3d(args.grid) if args.matrix == "laplacian" else W.graph_laplacian(args.n, seed=3)
        n = A.n
        rp = torch.as_tensor(A.indptr, device="cuda")
        ci = torch.as_tensor(A.indices, device="cuda")
        vals = torch.as_tensor(A.data, device="cuda")
        dt = {"df64": L.EIG_DF64, "f64": L.EIG_F64, "f32": L.EIG_F32}[args.arith]
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
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    status = L.device_status()
    print(json.dumps({"kernel": args.kernel, "arith": args.arith, "n": n, "a": a, "b": b, "sym": args.sym,
                      "ms": ms, "flops": flops, "bytes": nbytes, "tflops": flops / ms / 1e9,
                      "gbs": nbytes / ms / 1e6 if nbytes else None, "device_status": status}), flush=True)
    return 0 if status == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--strategy", default="fix")
    ap.add_argument("--form", default=None, choices=["f64", "df64", "mixed"],
                    help="block format (default: f64; mixed for the serving stream c5)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the solves under the other strategies (fixed block, slope, slopek)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--requests", type=int, default=32, help="c5: requests replayed from the stream")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="c5: device memory for active solves")
    ap.add_argument("--max-active", type=int, default=64, help="c5: solves advanced per step")
    ap.add_argument("--gram-tc", type=int, default=None, choices=[0, 1],
                    help="1 (default): Gram and update on the tensor cores (exact slices); 0: on the CUDA "
                         "cores")
    ap.add_argument("--tc-chunk-rows", type=int, default=None,
                    help="rows of the tensor-core slice buffers (a multiple of 128; products run over "
                         "row chunks; default: all rows, and 2^20 for c4, whose full slice buffers would "
                         "not fit in HBM)")
    ap.add_argument("--expand", default="drop", choices=["drop", "powered", "random"],
                    help="vectors appended at an expansion (Sec. 6.4): the saved ones, the saved ones "
                         "filtered every iteration (Chebyshev SI only), fresh Gaussian ones")
    ap.add_argument("--ablate-expand", action="store_true",
                    help="also solve once with each other expansion variant of Sec. 6.4")
    ap.add_argument("--aggressive-warmup", action="store_true",
                    help="warm-up gate on the first pair's residual with r_warm = 1e-1 (the paper's closing "
                         "remarks) instead of r^(j) <= 1e-4")
    ap.add_argument("--max-iter", type=int, default=1000,
                    help="iteration cap per solve (profiling runs use a small cap)")
    ap.add_argument("--ref-iters", type=int, default=315,
                    help="iterations per solve used to scale the reference arm's per-iteration time")
    ap.add_argument("--kernel", choices=["gram", "update", "spmm", "syev"],
                    help="time one kernel class instead of whole solves (--n, --a, --b, --sym, --arith, --grid)")
    ap.add_argument("--n", type=int, default=2097152)
    ap.add_argument("--a", type=int, default=384)
    ap.add_argument("--b", type=int, default=384)
    ap.add_argument("--sym", action="store_true")
    ap.add_argument("--grid", type=int, default=128, help="--kernel spmm: 3D Laplacian grid side")
    ap.add_argument("--matrix", default="laplacian", choices=["laplacian", "graph"],
                    help="--kernel spmm: the 3D Laplacian (--grid) or the power-law graph Laplacian of "
                         "the c4 workload with --n rows")
    ap.add_argument("--arith", default="f64_tc", choices=["df64", "df64_tc", "f64", "f64_tc", "f32", "c32"])
    args = ap.parse_args()
    if args.kernel:
        return run_kernel(args)
    if args.form is None:
        args.form = "mixed" if args.workload == "c5" else "f64"
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    if args.workload == "c5":
        return run_serving(args)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2409_05572_gb300 import _lib as L
    L.load()

    wl = make_workload(args.workload)
    A, nev, k, normA, tol = wl["A"], wl["nev"], wl["k_max"], wl["normA"], wl["tol"]
    X0 = W.gaussian_block(A.n, k, wl["seed"])
    dev = torch.device("cuda", local)
    rp = torch.as_tensor(A.indptr, device=dev)
    ci = torch.as_tensor(A.indices, device=dev)
    va = torch.as_tensor(A.data, device=dev)
    X0d = torch.as_tensor(X0, device=dev)
    stream = torch.cuda.Stream(device=dev)
    # stopping test of Eq. conv at tol/2 so that ||Av - lv|| / ||A|| <= tol holds
    algo = wl.get("algo", "lobpcg")
    extra = dict(wl.get("extra", {}))
    if args.gram_tc is not None:
        extra["gram_tc"] = args.gram_tc
    if args.tc_chunk_rows is not None:
        extra["tc_chunk_rows"] = args.tc_chunk_rows
    if args.aggressive_warmup:
        extra.update(warm_first=1, r_warm=1e-1)
    extra.update(EXPAND_OPTS[args.expand])
    solver = L.Solver((rp, ci, va), nev=nev, k_max=k, strategy=args.strategy, X0=X0d, normA=normA,
                      tol=0.5 * tol, form=args.form, stream=stream, profile=1, max_iter=args.max_iter,
                      algo=algo, **extra)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        out = solver.solve()
    barrier()
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kst = None
    results = []
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            out = solver.solve()
            results.append(out)
            ks = out["kstats"]
            if kst is None:
                kst = {c: dict(v) for c, v in ks.items()}
            else:
                for c, v in ks.items():
                    for f in v:
                        kst[c][f] += v[f]
        ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_step = reduce_step_time(ms_total / args.steps, dist, dev)
    value = job_value(nev, ws, ms_step)
    last = results[-1]
    ok = last["status"] == 0 and float(np.max(last["resid"])) <= tol
    eig_err = (float(np.max(np.abs(last["lam"] - wl["exact"]) / np.abs(wl["exact"])))
               if wl.get("exact") is not None else None)

    tc_on = extra.get("gram_tc", 1) != 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.form, "data": "synthetic",
            "config": {"workload": wl["desc"], "nev": nev, "k_max": k, "strategy": args.strategy,
                       "form": args.form, "tol": tol, "parallelism": f"replicas x{ws}",
                       "products": ("tensor cores (tcgen05, exact bf16 slices: "
                                    + ("7 slices, 28 pairs per float64 multiply-add)" if args.form == "f64"
                                       else "6 slices, 21 pairs per double-float multiply-add)"))
                       if tc_on else "CUDA cores",
                       "tc_chunk_rows": extra.get("tc_chunk_rows", 0),
                       "l2": f"inputs larger than L2 (each n x k_max block is {8 * A.n * k / 1e9:.1f} GB); no flush",
                       "warmup_rule": "first pair, r_warm 1e-1" if args.aggressive_warmup else "r^(j), r_warm 1e-4",
                       "expand": args.expand},
            "converged": bool(ok), "iters": last["iters"], "n_shrink": last["n_shrink"],
            "n_expand": last["n_expand"], "max_resid": float(np.max(last["resid"])),
            "max_rel_eig_err_vs_closed_form": eig_err, "clocks": clk}

    # per-kernel-class time shares and the roofline of the dominant kernel
    tot_ms = sum(v["ms"] for v in kst.values())
    line["kernel_share"] = {c: round(v["ms"] / tot_ms, 4) for c, v in kst.items() if v["launches"]}
    line["gpu_launches"] = int(sum(r["launches"] for r in results) / args.steps)
    hbm, _, src = peaks()
    dom = max(kst, key=lambda c: kst[c]["ms"])
    v = kst[dom]
    if dom == "spmm":
        ach = v["bytes"] / (v["ms"] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_source": src}
    elif dom in ("gram", "update") and tc_on and args.form in TC_MMA_PER_MAC:
        # tensor-core products: the bf16 MMA work the sliced method performs
        # (28 or 21 slice products per multiply-add of the method) against
        # the sustained bf16 peak; the class time includes the slicing passes
        per = TC_MMA_PER_MAC[args.form]
        alg = v["flops"] / (v["ms"] / 1e3) / 1e12
        ach = per * alg
        pk, psrc = bf16_sustained()
        roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "peak_source": psrc,
                "method_tflops": alg,
                "method_bytes_frac_of_hbm": v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm,
                "note": f"achieved = {per} bf16 slice products per {args.form} multiply-add x the method's "
                        "multiply-adds / class time (slicing passes included); method_tflops is the "
                        f"{args.form} rate of the method itself"}
    else:
        ach = v["flops"] / (v["ms"] / 1e3) / 1e12
        pk = FP64_PEAK_TFLOPS if args.form == "f64" else DF64_PEAK_TFLOPS
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk,
                "peak_source": "derived: FP32 issue rate measured on GB300 (36.3e12 FFMA/s) / "
                               "11.1 FP32 instructions per double-float multiply-add x 2"
                if args.form != "f64" else "measured native FP64 FMA rate"}
    roof["avg_launch_ms"] = v["ms"] / max(v["launches"], 1)
    if dom in TC_TRAFFIC_RATIO and tc_on and args.form == "f64":
        # per launch, like achieved: algorithmic bytes of the class's average
        # launch x the DRAM/algorithmic ratio of the ncu capture
        roof["traffic"] = TC_TRAFFIC_RATIO[dom] * v["bytes"] / max(v["launches"], 1)
        roof["traffic_source"] = (f"ncu dram__bytes_read+write of the {dom} class's kernels at n=262144 "
                                  f"(ratio {TC_TRAFFIC_RATIO[dom]:.2f} to algorithmic bytes), scaled")
    else:
        roof["traffic"] = None
    line["roofline"] = roof
    sp = kst.get("spmm")
    if sp and sp["launches"]:
        a = sp["bytes"] / (sp["ms"] / 1e3) / 1e9
        f = sp["flops"] / (sp["ms"] / 1e3) / 1e12
        # bytes of one row of V read per nonzero (element size of the class's
        # dominant format): the traffic of a gather without reuse, the bound
        # that applies when V is far larger than L2 and the column indices
        # are scattered (the power-law graph); the Laplacian reuses V rows
        # through L2 and reads V about once
        esz = 4 if args.form == "mixed" else 8
        g = sp["flops"] / 2 * esz / (sp["ms"] / 1e3) / 1e9
        line["spmm"] = {"hbm_gbs": a, "hbm_frac": a / hbm, "gather_gbs": g, "gather_frac": g / hbm,
                        "fp64_tflops": f if args.form == "f64" else None,
                        "fp64_pipe_frac": f / FP64_PEAK_TFLOPS if args.form == "f64" else None}

    if rank == 0 and not args.no_compare:
        # every other strategy once on the same workload and form; `none` is
        # the fixed block of k_max columns (the metric's comparison)
        strat = {args.strategy: {"value": value, "ms": ms_step, "iters": last["iters"],
                                 "n_shrink": last["n_shrink"], "n_expand": last["n_expand"], "converged": bool(ok)}}
        for name in ("none", "fix", "slope", "slopek"):
            if name in strat:
                continue
            other = L.Solver((rp, ci, va), nev=nev, k_max=k, strategy=name, X0=X0d, normA=normA, tol=0.5 * tol,
                             form=args.form, stream=stream, max_iter=args.max_iter, algo=algo, **extra)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fo = other.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            fms = e0.elapsed_time(e1)
            fconv = bool(fo["status"] == 0 and np.max(fo["resid"]) <= tol)
            # a solve stopped by the iteration cap has no time-to-converged-nev
            strat[name] = {"value": nev / (fms / 1e3) if fconv else None, "ms": fms, "iters": fo["iters"],
                           "n_shrink": fo["n_shrink"], "n_expand": fo["n_expand"], "converged": fconv}
            other.close()
        line["strategies"] = strat
        fb = strat["none"]
        line["fixed_block"] = {"value": fb["value"], "unit": UNIT, "ms": fb["ms"], "iters": fb["iters"],
                               "converged": fb["converged"],
                               "speedup_of_shrink_expand": fb["ms"] / ms_step if fb["converged"] and ok else None}

    if rank == 0 and args.ablate_expand:
        # the vectors appended at an expansion (Sec. 6.4): each other variant
        # once, same workload, strategy and form
        var = {args.expand: {"ms": ms_step, "iters": last["iters"], "n_expand": last["n_expand"],
                             "converged": bool(ok)}}
        for name in ("drop", "powered", "random"):
            if name in var or (name == "powered" and algo != "chebsi"):
                continue
            ex2 = dict(extra)
            ex2.update(expand_powered=0, expand_random=0)
            ex2.update(EXPAND_OPTS[name])
            other = L.Solver((rp, ci, va), nev=nev, k_max=k, strategy=args.strategy, X0=X0d, normA=normA,
                             tol=0.5 * tol, form=args.form, stream=stream, max_iter=args.max_iter, algo=algo,
                             **ex2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fo = other.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            var[name] = {"ms": e0.elapsed_time(e1), "iters": fo["iters"], "n_expand": fo["n_expand"],
                         "converged": bool(fo["status"] == 0 and np.max(fo["resid"]) <= tol)}
            other.close()
        line["expand_variants"] = var

    if rank == 0 and not args.no_e2e:
        # end to end through the public API: host CSR + pinned host X0 in,
        # eigenvalues and eigenvectors back to the host
        X0h = torch.as_tensor(X0).pin_memory()
        Vh = torch.empty(A.n, nev, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = L.Solver(A, nev=nev, k_max=k, strategy=args.strategy, X0=X0h.numpy(), normA=normA, tol=0.5 * tol,
                      form=args.form, stream=stream, max_iter=args.max_iter, algo=algo, **extra)
        o2 = s2.solve()
        Vd = s2.V()
        Vh.copy_(Vd)
        torch.cuda.synchronize()
        s2.close()
        t_e2e = time.perf_counter() - t0
        h2d = A.indptr.nbytes + A.indices.nbytes + A.data.nbytes + X0.nbytes
        line["e2e"] = {"value": nev / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(Vh.numel() * 8 + nev * 8), "seconds": t_e2e}

    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, args.strategy, last["iters"])

    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
