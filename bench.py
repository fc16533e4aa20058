#!/usr/bin/env python
"""Benchmark of the FP64 supernodal Cholesky factorization + solve on one GB300 per rank.

Workload (default): 3D 27-point stencil, 3 unknowns per node, 80^3 grid (n = 1,536,000),
nested-dissection ordering, seed 5, FP64 -- the largest single-GPU configuration; one
step = numeric factorization (all levels: assembly, POTRF, TRSM, Schur update + scatter)
+ one forward/back solve with b = A x_true.  Inputs (values, right-hand side) are resident
in HBM before the timed region; the factor (33 GB) and the values are far larger than L2,
so no flush is needed.

value     = factorization flops (sum_j c_j^2) per second of the whole step, all ranks
e2e       = the same through the C ABI with host (pinned) buffers: values and b copied in,
            x copied out, every step
roofline  = the dominant kernel's algorithmic work / its CUDA-event time inside the timed
            region (events bracket that kernel kind alone, so the other launches carry no
            event overhead), against its peak; the kernel shares come from a separate pass
            with every launch bracketed

Multi-GPU: one process per GPU (torchrun), each factoring its own replica (the
factorization of one matrix is not sharded): weak scaling, no data-path collective.
``--impl reference`` times the CPU oracle (test code, single thread) on a bounded
sample of the same family instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor GFLOP/s + % FP64 peak; served solves/s and p99 latency at resid<=1e-12"
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0  # nominal dense FP64 / BF16 rates of a GB300
FALLBACK_BF16_TFLOPS = 1900.0
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
OZ_PRODUCTS = 36  # slice pairs p + q < 8 of the FP64 tensor-core Schur tiles
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 rates of a GB300



GRANULARITY = {"tiles": 0, "optd": 1, "optd_cost": 2, "hybrid": 3}

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"bf16_tflops": FALLBACK_BF16_TFLOPS, "hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.split(",") for r in f.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ("factor_kernels.cu", "oz_kernels.cu", "tc_kernels.cu", "device_common.cuh",
                  "chol_internal.h")
# the source files that define each traced kernel kind (its device code and shared helpers)
KIND_SOURCES = {"schur128_oz": ("oz_kernels.cu", "device_common.cuh"),
                "schur128_tc": ("tc_kernels.cu", "device_common.cuh")}


def kernel_source_hash(kind: str | None = None) -> str:
    """Hash of the device sources of a kernel kind (all kernel sources if unknown): a stored
    ncu traffic figure is used only while the kernel it was measured on is unchanged."""
    h = hashlib.sha256()
    for f in KIND_SOURCES.get(kind, KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_2202_09288_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, flops_per_launch: float):
    """DRAM bytes per launch of `kernel`: the committed ncu capture's bytes per
    algorithmic flop (a smaller case of the same kernel) times this launch size's flops,
    provided the capture was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e["dram_bytes_per_flop"] * flops_per_launch


def oracle_sample(name: str):
    """Times the CPU oracle (one thread) on one factorization + solve of a sample."""
    import oracle
    from paper_2202_09288_gb300 import inputs

    A, perm = inputs.workload(name)
    bp, bi, bx = oracle.permute(A.n, A.colptr, A.rowind, A.vals, perm)
    parent, cc, lp, li = oracle.symbolic(A.n, bp, bi)
    b = A.to_scipy_full() @ inputs.rhs_block(1, A.n, 1)[:, 0]
    t0 = time.perf_counter()
    lx, fl = oracle.factor(A.n, bp, bi, bx, lp, li)
    x = oracle.solve(A.n, lp, li, lx, perm, b)
    dt = time.perf_counter() - t0
    flops = float(np.sum(cc.astype(np.float64) ** 2))
    return flops, dt, x


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest x over all ranks: the timed region is the slowest rank's.  dist is
    torch.distributed (any backend; device "cuda" for NCCL, "cpu" for gloo) or None."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, flops_per_rank: float, seconds: float) -> float:
    """Whole-job GFLOP/s of `world` independent replicas (weak scaling: every rank factors
    its own matrix of flops_per_rank), over the slowest rank's time."""
    return world * flops_per_rank / seconds / 1e9


def tasks_sample(name: str, width: int, relax: float):
    """Times the multi-core CPU baseline of the paper's tasking (left-looking supernodal
    factorization as OpenMP tasks, Sec. 3 and 4) on all host cores, one factorization per
    policy (best of two), on the same sample and supernode partition as the GPU path."""
    import cpu_tasks
    import paper_2202_09288_gb300 as P
    from paper_2202_09288_gb300 import inputs

    A, perm = inputs.workload(name)
    sym = P.Symbolic(P.make_opts(width_cap=width, relax=relax), A, perm)
    rowptr, rows = P.chol_sym_rows(sym.handle)
    start = sym.export()["sn_start"]
    F = sym.info["flops"]
    cores = os.cpu_count() or 1
    out = {}
    for pol in cpu_tasks.POLICIES:
        best, D, inner = float("inf"), -1, 0
        for _ in range(2):
            pan = cpu_tasks.factor(A, perm, start, rowptr, rows, pol, threads=cores)
            best, D, inner = min(best, pan.seconds), pan.D, pan.inner_tasks
        out[pol] = {"gflops": F / best / 1e9, "seconds": best, "D": D, "inner_tasks": inner}
    return {"value": out["optd_cost"]["gflops"], "unit": "GFLOP/s", "cores": cores,
            "kind": "paper tasking (OPT-D-COST, OpenMP, plain-loop dense kernels)",
            "sample": f"{name}: one FP64 factorization ({F:.3e} flops) per policy, best of 2",
            "policies": out}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    sample = args.ref_sample
    times, flops = [], 0.0
    for i in range(args.warmup + args.steps):
        flops, dt, _ = oracle_sample(sample)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    gf = flops / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gf, "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": gf, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample}: one FP64 factorization + 1-RHS solve per step "
                                   f"({flops:.3e} flops) by the single-thread C oracle"},
        "e2e": {"value": gf, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_batched(args):
    """Plain per-level launches vs autotuned tiles vs a CUDA-graph batch (one matrix), and a
    batch of several matrices vs factoring them one after another."""
    import torch

    import paper_2202_09288_gb300 as P
    from paper_2202_09288_gb300 import inputs

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = P.Context(width_cap=args.width, stream=stream.cuda_stream)
    prec = P.CHOL_MIXED if args.precision == "mixed" else P.CHOL_FP64
    A, perm = inputs.workload(args.workload)
    sym = P.Symbolic(ctx, A, perm)
    F = sym.info["flops"]
    vals_d = torch.from_numpy(A.vals).cuda()
    torch.cuda.synchronize()
    num = P.Factor(ctx, sym, vals_d, precision=prec)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 1)):
            fn()
        e0, e1 = _events(torch, 2)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    plain_ms = timed(lambda: num.refactor(vals_d), args.steps)
    default_policy = P.chol_sym_get_tile_policy(sym.handle)
    policy, _ = num.autotune(reps=1)
    tuned_ms = timed(lambda: num.refactor(vals_d), args.steps)
    batch = P.Batch(ctx, [num])
    graph_ms = timed(lambda: batch.factorize(use_graph=True), args.steps)
    assert num.status()[0] == P.CHOL_OK
    batch.close()
    # several matrices of one family: one after another vs one batch (graph replay)
    mname, mcount = args.multi.split(":")
    mcount = int(mcount)
    M, mperm = inputs.workload(mname)
    msym = P.Symbolic(ctx, M, mperm)
    mvals = [torch.from_numpy(M.vals * (1.0 + 0.1 * i)).cuda() for i in range(mcount)]
    torch.cuda.synchronize()
    mnums = [P.Factor(ctx, msym, v, precision=prec) for v in mvals]
    seq_ms = timed(lambda: [f.refactor(v) for f, v in zip(mnums, mvals)], args.steps)
    mbatch = P.Batch(ctx, mnums)
    mb_ms = timed(lambda: mbatch.factorize(use_graph=True), args.steps)
    ok = all(f.status()[0] == P.CHOL_OK for f in mnums)
    mbatch.close()
    MF = msym.info["flops"] * mcount
    line = {
        "metric": METRIC, "mode": "batched", "value": F / (graph_ms * 1e-3) / 1e9,
        "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": graph_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == P.CHOL_MIXED else "f64",
        "data": "synthetic",
        "config": dict(workload_config(args), n=A.n, flops_per_step=F,
                       nlevels=sym.info["nlevels"]),
        "plain_per_level_ms": plain_ms, "autotuned_ms": tuned_ms, "graph_batch_ms": graph_ms,
        "default_tile_policy": default_policy, "autotuned_tile_policy": policy,
        "multi": {"matrix": mname, "count": mcount, "sequential_ms": seq_ms,
                  "batched_graph_ms": mb_ms, "speedup": seq_ms / mb_ms,
                  "batched_gflops": MF / (mb_ms * 1e-3) / 1e9, "all_ok": ok},
    }
    print(json.dumps(line))
    return 0


def serve_requests(count, seed):
    """The serving workload: 2D 5-point or 3D 7-point SPD systems (probability 1/2 each)
    with n log-uniform in [1e3, 2e5] (k = round(sqrt n) or round(cbrt n)), a diagonal shift
    sigma ~ U[0, 1) times the diagonal (new values on a shared pattern), 1-8 right-hand sides
    with b = A x_true, x_true ~ U[-1, 1) (one block of 8 per pattern)."""
    from paper_2202_09288_gb300 import inputs

    u = (inputs.uniform(seed, 12, 4 * count) + 1.0) / 2.0
    patterns = {}
    out = []
    for r in range(count):
        n = math.exp(math.log(1e3) + u[4 * r + 1] * (math.log(2e5) - math.log(1e3)))
        if u[4 * r] < 0.5:
            key = ("lap2d", max(2, round(n ** 0.5)))
        else:
            key = ("diff3d7", max(2, round(n ** (1.0 / 3.0))))
        if key not in patterns:
            A, perm = inputs.workload(f"{key[0]}_{key[1]}")
            patterns[key] = (A, perm, A.to_scipy_full(), A.vals[A.colptr[:-1]],
                             inputs.rhs_block(seed * 1000 + len(patterns), A.n, 8))
        A, perm, Afull, diag, Xp = patterns[key]
        sigma = u[4 * r + 2]
        vals = A.vals.copy()
        vals[A.colptr[:-1]] *= 1.0 + sigma
        Ar = inputs.SpdMatrix(A.n, A.colptr, A.rowind, vals, A.grid, A.dofs)
        nrhs = 1 + min(7, int(8 * u[4 * r + 3]))
        X = Xp[:, :nrhs]
        B = np.asfortranarray(Afull @ X + (sigma * diag)[:, None] * X)  # (A + sigma D) X
        out.append((Ar, perm, B))
    return out


def run_serve(args):
    """Request stream through the server: closed loop (all requests queued at once) for
    throughput, then Poisson arrivals at 0.5 and 0.9 of that throughput for latency."""
    import threading

    import torch  # noqa: F401  (CUDA context of this process)

    import paper_2202_09288_gb300 as P
    from paper_2202_09288_gb300 import inputs

    prec = P.CHOL_MIXED if args.precision == "mixed" else P.CHOL_FP64
    reqs = serve_requests(args.requests, 4)
    srv = P.Server(slots=2, max_batch=16, hbm_budget=64 << 30, width_cap=args.width)
    # warm-up: module load, analysis caches of the first patterns
    for t in [srv.submit(A, p, B, precision=prec, tol=args.tol) for A, p, B in reqs[:20]]:
        srv.wait(t)

    def run(arrivals):
        """arrivals: None (all at once) or submit times relative to the start."""
        tickets = [None] * len(reqs)
        start = srv.clock()

        def submitter():
            for i, (A, p, B) in enumerate(reqs):
                if arrivals is not None:
                    dt = start + arrivals[i] - srv.clock()
                    if dt > 0:
                        time.sleep(dt)
                tickets[i] = srv.submit(A, p, B, precision=prec, tol=args.tol)

        th = threading.Thread(target=submitter)
        th.start()
        th.join() if arrivals is None else None
        res = []
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(1e-4)
            res.append(srv.wait(tickets[i])[1])
        th.join()
        return res

    closed = run(None)
    t_first = min(r["t_submit"] for r in closed)
    t_last = max(r["t_done"] for r in closed)
    span = t_last - t_first
    rate = len(reqs) / span
    solves = sum(B.shape[1] for _, _, B in reqs)
    out = {"closed_loop": {"requests": len(reqs), "seconds": span, "requests_per_s": rate,
                           "solves_per_s": solves / span}}
    for load in (0.5, 0.9):
        lam = load * rate
        uu = (inputs.uniform(40 + int(load * 10), 13, len(reqs)) + 1.0) / 2.0
        gaps = -np.log(np.maximum(uu, 1e-300)) / lam
        arr = np.cumsum(gaps) - gaps[0]
        res = run(list(arr))
        lat = np.array([r["t_done"] - r["t_submit"] for r in res])
        span_o = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
        out[f"poisson_{load}"] = {
            "arrival_rate_per_s": lam, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean([r["batch_size"] for r in res])),
            "solves_per_s": solves / span_o,
            "max_residual": float(max(r["residual"] for r in res)),
            "failed": int(sum(r["status"] != 0 for r in res))}
    srv.close()
    allres = closed
    line = {
        "metric": METRIC, "mode": "serve", "value": out["closed_loop"]["solves_per_s"],
        "unit": "solves/s", "n_gpus": 1, "steps": len(reqs), "warmup": 20,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == P.CHOL_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "serving stream: 2D 5-pt / 3D 7-pt, n log-uniform [1e3, 2e5], "
                               "1-8 RHS, 64 GB budget, 2 slots, groups of <= 16",
                   "precision": args.precision, "tol": args.tol},
        "p50_ms": out["poisson_0.9"]["p50_ms"], "p99_ms": out["poisson_0.9"]["p99_ms"],
        "max_residual": float(max(r["residual"] for r in allres)),
        "failed": int(sum(r["status"] != 0 for r in allres)),
        **out,
    }
    print(json.dumps(line))
    return 0


def workload_config(args, l_storage=None):
    size = (f"factor {l_storage * (4 if args.precision == 'mixed' else 8) / 1e9:.1f} GB"
            if l_storage else "factor of several GB")
    return {"workload": args.workload, "n": None, "precision": args.precision,
            "nrhs": args.nrhs,
            "ordering": "geometric nested dissection (leaf 64 nodes)",
            "width_cap": args.width, "assembly": args.assembly,
            "fp64_schur": getattr(args, "fp64_schur", "ozaki"),
            "l2": f"inputs larger than L2 ({size}), no flush"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="st27x3_80")
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--assembly", default="atomic", choices=["atomic", "owner"])
    ap.add_argument("--cpu-sample", default="st27x3_24")
    ap.add_argument("--ref-sample", default="st27x3_20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: FP32 factor + FP64 iterative refinement to --tol")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--policy", default="",
                    help="Schur tile policy overrides as JSON, e.g. "
                         "'{\"min_rows_tile128\": 1073741824}' (no 128-wide tiles)")
    ap.add_argument("--granularity", default="tiles", choices=list(GRANULARITY),
                    help="Schur task granularity: size thresholds alone (tiles), or the paper's "
                         "OPT-D / OPT-D-COST / hybrid rules applied to the tiles")
    ap.add_argument("--fp64-schur", default="ozaki", choices=["ozaki", "dmma"],
                    help="FP64 128-wide Schur tiles: bf16 tensor-core slices or FP64 DMMA")
    ap.add_argument("--relax", type=float, default=0.0,
                    help="relaxed amalgamation zero share (0: library default, <0: off)")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--mode", default="factor", choices=["factor", "batched", "serve"],
                    help="factor: one matrix per step (default); batched: plain per-level "
                         "launches vs autotuned tiles vs CUDA-graph batches; serve: request "
                         "stream through the server")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=10,
                    help="steps of the end-to-end (host buffer) measurement (at most --steps)")
    ap.add_argument("--trace-steps", type=int, default=2,
                    help="steps of the separate fully traced pass (kernel shares)")
    ap.add_argument("--multi", default="st27x3_24:8",
                    help="batched mode: name:count of the multi-matrix batch")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "serve":
        return run_serve(args)

    import torch

    import paper_2202_09288_gb300 as P
    from paper_2202_09288_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    A, perm = inputs.workload(args.workload)
    n = A.n
    nrhs = args.nrhs
    Xt = inputs.rhs_block(1, n, nrhs)
    Afull = A.to_scipy_full()
    b = np.asfortranarray(Afull @ Xt)
    mixed = args.precision == "mixed"
    prec = P.CHOL_MIXED if mixed else P.CHOL_FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = P.Context(device=local, width_cap=args.width,
                    assembly=P.CHOL_ASSEMBLY_OWNER if args.assembly == "owner"
                    else P.CHOL_ASSEMBLY_ATOMIC, stream=stream.cuda_stream,
                    relax=args.relax,
                    fp64_schur=P.CHOL_SCHUR_DMMA if args.fp64_schur == "dmma"
                    else P.CHOL_SCHUR_OZAKI)
    sym = P.Symbolic(ctx, A, perm)
    if args.policy:
        P.chol_sym_set_tile_policy(sym.handle, json.loads(args.policy))
    if args.granularity != "tiles":
        P.chol_sym_set_tile_policy(sym.handle, {"granularity": GRANULARITY[args.granularity]})
    F = sym.info["flops"]
    vals_d = torch.from_numpy(A.vals).cuda()
    b_d = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()  # (k, n): column c = row c
    x_d = torch.empty_like(b_d)
    torch.cuda.synchronize()
    num = P.Factor(ctx, sym, vals_d, precision=prec)
    refine_info = {}

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        num.refactor(vals_d)
        if ev is not None:
            ev[1].record(stream)
        if mixed:
            _, info = num.refine(b_d, x_d, tol=args.tol)
            refine_info.update(info)
        else:
            num.solve(b_d, x_d)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    rc, bad = num.status()
    if rc != P.CHOL_OK:
        raise SystemExit(f"factorization failed: {P.chol_strerror(rc)} at column {bad}")

    # kernel shares: a separate pass with every launch bracketed by events
    P.chol_profile_reset(ctx.handle)
    P.chol_profile_only(ctx.handle, None)
    P.chol_profile_enable(ctx.handle, True)
    for _ in range(max(args.trace_steps, 1)):
        step()
    torch.cuda.synchronize()
    P.chol_profile_enable(ctx.handle, False)
    traced = P.chol_profile_read(ctx.handle)
    trace_steps = max(args.trace_steps, 1)
    fac_kinds = {kk: v for kk, v in traced.items() if v["timed"] > 0 and v["flops"] > 0}
    dom = max(fac_kinds, key=lambda kk: fac_kinds[kk]["ms"])

    # the timed region: events bracket the dominant kernel kind only
    clocks = ClockSampler(local)
    P.chol_profile_reset(ctx.handle)
    P.chol_profile_only(ctx.handle, dom)
    P.chol_profile_enable(ctx.handle, True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for it in range(args.steps):
        step(evs[it])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    P.chol_profile_enable(ctx.handle, False)
    P.chol_profile_only(ctx.handle, None)
    prof = P.chol_profile_read(ctx.handle)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), dist, "cuda")
    ms_step = total_ms / args.steps
    fac_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    sol_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    x = np.asfortranarray(x_d.cpu().numpy().T)
    anorm = np.abs(Afull).sum(axis=1).max()
    resid = float(max(np.abs(b[:, c] - Afull @ x[:, c]).max() / (anorm * np.abs(x[:, c]).max())
                      for c in range(nrhs)))
    launches = sum(v["launches"] for v in prof.values())

    # end to end through host buffers (pinned): values + b in, x out, every step
    vals_h = torch.empty(A.vals.shape, dtype=torch.float64, pin_memory=True).numpy()
    vals_h[:] = A.vals
    b_h = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).numpy().T
    b_h[:] = b
    x_h = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).numpy().T

    def host_step():
        num.refactor(vals_h)
        if mixed:
            info = P.chol_refine_info()
            rc = P.lib().chol_refine(ctx.handle, num.handle, nrhs, b_h.ctypes.data, n,
                                     x_h.ctypes.data, n, P.CHOL_HOST, args.tol, 10, info)
            if rc:
                raise P.CholError(rc, "chol_refine")
        else:
            P.chol_solve(ctx.handle, num.handle, b_h, x_h)

    host_step()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")

    peaks, peak_src = measured_peaks()
    fp64_peak_tflops = peaks["bf16_tflops"] * NOMINAL_FP64_OVER_BF16
    d = prof[dom]  # the dominant kind, bracketed alone inside the timed region
    achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
    traffic = ncu_traffic(dom, d["flops"] / max(d["timed"], 1))
    if dom == "schur128_oz":
        # FP64 tiles on the bf16 tensor cores: 36 bf16 slice products per FP64 product
        achieved *= OZ_PRODUCTS
        roof = {"bound": "tensor", "peak": peaks["bf16_tflops"],
                "peak_source": f"bf16 tensor {peak_src} {peaks['bf16_tflops']} TFLOP/s; achieved "
                               f"= {OZ_PRODUCTS} bf16 slice products x the tiles' FP64 flops / "
                               "time (FP64-equivalent rate = achieved / 36)"}
    elif dom == "schur128_tc":
        # FP32 tiles on the TF32 tensor cores: three TF32 products per FP32 product
        achieved *= 3
        tf32_peak = peaks["bf16_tflops"] * NOMINAL_TF32_OVER_BF16
        roof = {"bound": "tensor", "peak": tf32_peak,
                "peak_source": f"TF32 = {peak_src} bf16 {peaks['bf16_tflops']} TFLOP/s x nominal "
                               "TF32/bf16 1.1/2.25; achieved = 3 TF32 products (3xTF32) x the "
                               "tiles' FP32 flops / time"}
    elif dom.endswith("_f64"):
        roof = {"bound": "tensor", "peak": fp64_peak_tflops,
                "peak_source": f"FP64 = {peak_src} bf16 {peaks['bf16_tflops']} TFLOP/s x "
                               "nominal FP64/bf16 1.25/2250 (DMMA loop measured 1.046 "
                               "TFLOP/s on this pool)"}
    else:
        roof = {"bound": "alu", "peak": FP32_SIMT_PEAK_TFLOPS,
                "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 "
                               "TFLOP/s nominal; 72.0 measured by an FFMA loop"}

    # the step's solve against HBM: each pass reads every stored value of L once (the
    # diagonal blocks as their inverses' lower triangles, the same count) plus the vectors
    esz = 4 if mixed else 8
    solve_bytes = 2.0 * esz * sym.info["nnz_l"] + 2.0 * 3 * 8 * n * nrhs
    solve_roof = {"bound": "hbm", "achieved": solve_bytes / (sol_ms * 1e-3) / 1e9,
                  "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": solve_bytes / (sol_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                  "bytes": solve_bytes, "ms": sol_ms,
                  "note": f"2 passes x {esz} B x nnz(L) + vectors; solve time from the timed "
                          "region's CUDA events" + (" (refinement included)" if mixed else "")}
    if not mixed:
        # the same solve against the FP64 unit: one FP64 FMA per stored value of L per pass
        # and right-hand side, which on this part bounds the solve before HBM does
        solve_flops = 2.0 * 2.0 * sym.info["nnz_l"] * nrhs
        solve_roof["fp64"] = {"achieved": solve_flops / (sol_ms * 1e-3) / 1e12,
                              "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                              "frac": solve_flops / (sol_ms * 1e-3) / 1e12 / fp64_peak_tflops,
                              "flops": solve_flops}
    value = replica_rate(world, F, ms_step * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else (
            "f64 (Schur tiles: exact bf16x8 splits on tensor cores)"
            if args.fp64_schur == "ozaki" and args.width <= 64 else "f64"),
        "data": "synthetic",
        "config": dict(workload_config(args, sym.info["l_storage"]), n=n, nnz_a=A.nnz_lower,
                       nnz_l=sym.info["nnz_l"],
                       flops_per_step=F, flops_panel=sym.info["flops_panel"],
                       nsuper=sym.info["nsuper"], nfundamental=sym.info["nfundamental"],
                       nlevels=sym.info["nlevels"],
                       tile_policy=P.chol_sym_get_tile_policy(sym.handle),
                       granularity=P.chol_sym_granularity(sym.handle),
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "factor_ms": fac_ms, "solve_ms": sol_ms, "solve_roofline": solve_roof,
        "factor_gflops": F / (fac_ms * 1e-3) / 1e9,
        "fp64_peak_frac": (F / (fac_ms * 1e-3) / 1e12) / fp64_peak_tflops,
        "residual": resid,
        "gpu_launches": int(launches),
        "e2e": {"value": replica_rate(world, F, e2e_s), "unit": "GFLOP/s", "steps": e2e_steps,
                "h2d_bytes_per_step": int(A.vals.nbytes + b_h.nbytes),
                "d2h_bytes_per_step": int(x_h.nbytes)},
        "roofline": {"bound": roof["bound"], "kernel": dom, "achieved": achieved,
                     "peak": roof["peak"], "unit": "TFLOP/s",
                     "frac": achieved / roof["peak"], "traffic": traffic,
                     "launches_timed": d["timed"], "ms_per_step": d["ms"] / args.steps,
                     "peak_source": roof["peak_source"]},
        "kernels": {k: {"launches": v["launches"] / trace_steps, "ms": v["ms"] / trace_steps,
                        "share": v["ms"] / max(sum(w["ms"] for w in traced.values()), 1e-9)}
                    for k, v in traced.items() if v["launches"]},
        "kernels_source": f"separate pass of {trace_steps} steps with every launch bracketed "
                          "by events (per step)",
        "clocks": clk,
    }
    if mixed:
        line["refine"] = refine_info
        # the FP64 factor of the same matrix, timed once, for comparison
        f64 = P.Factor(ctx, sym, vals_d, precision=P.CHOL_FP64)
        f64.status()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        f64.refactor(vals_d)
        e1.record(stream)
        f64.solve(b_d, x_d)
        e2.record(stream)
        torch.cuda.synchronize()
        line["fp64_reference"] = {"factor_ms": e0.elapsed_time(e1),
                                  "solve_ms": e1.elapsed_time(e2),
                                  "factor_gflops": F / (e0.elapsed_time(e1) * 1e-3) / 1e9}
        del f64
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fl, dt, _ = oracle_sample(args.cpu_sample)
        line["cpu_baseline"] = {
            "value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{args.cpu_sample}: one FP64 factorization + 1-RHS solve "
                      f"({fl:.3e} flops, {dt:.1f} s) by the single-thread C oracle"}
        line["cpu_tasks_baseline"] = tasks_sample(args.cpu_sample, args.width, args.relax)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
