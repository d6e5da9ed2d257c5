#!/usr/bin/env python
"""Benchmark: H2 construction throughput on one GB300.

One step = one full construction from device-resident points: KD tree and
block lists, then the adaptive-sketching build (fused kernel-summation sketch,
near field, QR convergence test with extra sample rounds, row IDs, couplings)
of the 3D covariance workload: 131072 points uniform in [0,1]^3, Matern-3/2
(l = 0.1) plus a 1e-4 nugget, leaf 64, eta 0.7, tol 1e-6.  The headline value
is points built per second for the mixed-precision path; the FP64 path, the
approximation error, the roofline of the dominant kernel (the fused sketch),
an end-to-end run through the C ABI with host buffers and the CPU oracle on a
bounded sample are reported beside it.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2 build time & points/s at tol, mixed vs FP64 on 1 GB300; % HBM/compute roofline"
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.55
FP64_PEAK_TFLOPS = 1.25
# The tensor-core sketch is bound by entry generation on the special-function
# units: a Matern-3/2 entry takes two of their operations (square root and
# exp2); 16 SFU lanes per SM (4 per sub-partition).
SFU_LANES, SFU_OPS_PER_PAIR = 16, 2
SFU_PEAK_GPAIRS = SMS * SFU_LANES * SM_MAX_MHZ * 1e6 / SFU_OPS_PER_PAIR / 1e9   # 2516.5
WORKLOAD_DESC = ("c2: N=131072 uniform [0,1]^3, Matern-3/2 l=0.1 + 1e-4 nugget, leaf 64, "
                 "eta 0.7, tol 1e-6, adaptive sampling up to 256 columns (schedule in config.schedule), "
                 "fused kernel-summation sketch")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(n_sample: int) -> dict:
    """Full oracle build of the same workload family at n_sample points.
    Runs in a child process with single-threaded BLAS (cores = 1)."""
    from oracle import h2_oracle as O
    from paper_2506_16759_gb300 import workloads as W
    w = W.scaled(W.config("c2"), n_sample)
    X = w.points()
    om = w.omega()
    t0 = time.perf_counter()
    t = O.build_cluster_tree(X, w.leaf_size)
    lists = O.dual_traversal(t, w.eta)
    t_tree = time.perf_counter() - t0
    h = O.build_h2(t, lists, w.kernel, w.params, w.tol, om,
                   O.ksum_sampler(X, w.kernel, w.params, 512), w.d0, w.d_inc, w.d_max)
    return {"n": n_sample, "t_tree": t_tree, "t_sketch": h.timings["sketch_s"],
            "t_construct": h.timings["construct_s"], "d_final": h.d_final}


def run_oracle_child(n_sample: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                          str(n_sample)], capture_output=True, text=True, env=env, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def scaled_oracle_rate(r: dict, n_full: int) -> tuple[float, float]:
    """Oracle seconds for the full workload from a sample: the sketch scales as
    N^2 (direct summation), tree and construction as N."""
    f = n_full / r["n"]
    secs = r["t_sketch"] * f * f + (r["t_construct"] + r["t_tree"]) * f
    return n_full / secs, secs


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"h2_bench_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("sketch.cu", "sketch_tc.cu", "h2_internal.cuh", "h2_ops.h"):
        h.update(open(os.path.join(ROOT, "paper_2506_16759_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(prec: str):
    """DRAM bytes per sketch launch from the committed ncu summary, if the
    kernel source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", f"ksum_tc_c2_{prec}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != source_hash():
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- ranks
# One process per GPU; each rank builds its own replica of the workload (no
# data-path collective).  These helpers are the only cross-rank steps: a
# barrier around the timed region and the maximum of the ranks' times.
RANK_TIMEOUT_S = 300   # a rank that dies makes the others' next collective fail


def rank_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(v: float, world: int, device=None) -> float:
    """Largest value over the ranks (every rank gets it)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, n_per_rank: int, steps: int, max_total_ms: float) -> float:
    """Points per second of the whole job: every rank built steps x n points
    and the job took the slowest rank's time."""
    return world * n_per_rank * steps / (max_total_ms / 1e3)


# ---------------------------------------------------------------- GPU arm
def main_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import _lib
    from paper_2506_16759_gb300 import workloads as W

    import datetime
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev,
                                timeout=datetime.timedelta(seconds=RANK_TIMEOUT_S))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # CPU oracle sample first (a child process; no fork of a CUDA process)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            r = run_oracle_child(args.cpu_sample)
            rate, secs = scaled_oracle_rate(r, W.config("c2").n)
            cpu = {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle",
                   "sample": (f"full oracle build of the same workload at N={r['n']} "
                              f"(sketch {r['t_sketch']:.1f}s, construction "
                              f"{r['t_construct']:.1f}s, tree {r['t_tree']:.1f}s, 1 thread); "
                              f"scaled to N=131072 as sketch*(N/n)^2 + rest*(N/n): "
                              f"{secs:.0f}s per build")}
        except Exception as e:  # the baseline must not sink the GPU line
            cpu = {"value": None, "unit": "points/s", "cores": 1, "kind": "oracle",
                   "sample": f"failed: {e}"}

    w = W.config("c2")
    X = torch.from_numpy(w.points()).to(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    prec = args.prec
    sched = {"d0": w.d0, "d_inc": w.d_inc, "prec": prec}
    tuned = None
    if args.autotune:
        # sample schedule and sketch engine picked by timed builds on this problem
        t0 = time.perf_counter()
        tree0 = api.ClusterTree(X, w.leaf_size, w.eta)
        kw, ms = api.autotune(tree0, w.kernel, w.params, w.tol, prec=prec, d0=w.d0,
                              d_inc=w.d_inc, d_max=w.d_max, seed=99)
        del tree0
        sched = {"d0": kw["d0"], "d_inc": kw["d_inc"], "prec": kw["prec"]}
        tuned = dict(sched, tuning_s=time.perf_counter() - t0, build_ms=ms)
        log(f"[bench] autotuned schedule {sched} ({ms:.1f} ms build)")

    def step(seed, precision, timing=True, schedule=None):
        sc = schedule or sched
        if precision == "fp64":
            sc = {"d0": w.d0, "d_inc": w.d_inc, "prec": "fp64"}
        tree = api.ClusterTree(X, w.leaf_size, w.eta)
        h = api.H2Matrix.build(tree, w.kernel, w.params, w.tol, prec=sc["prec"], seed=seed,
                               sketch="ksum", timing=timing, d0=sc["d0"], d_inc=sc["d_inc"],
                               d_max=w.d_max)
        return tree, h

    log(f"[bench] warmup {args.warmup} x {prec}")
    for i in range(args.warmup):
        step(1000 + i, prec)
    barrier()
    L = _lib.lib()
    clocks = ClockSampler(local) if rank == 0 else None
    launches0 = L.h2_kernel_launches()
    times = []
    for k in range(args.steps):
        flush.zero_()               # L2 flush between timed steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        tree, h = step(k, prec, timing=False)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        del h, tree
    barrier()
    launches = L.h2_kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    # phase breakdown and per-launch kernel times from instrumented builds of
    # the same problem, after the timed region (the phase timers synchronise)
    stats = []
    for k in range(2):
        flush.zero_()
        tree, h = step(k, prec, timing=True)
        stats.append(h.stats())
        del h, tree
    total_ms = max_over_ranks(sum(times), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, w.n, args.steps, total_ms)
    log(f"[bench] {prec}: {ms_per_step:.1f} ms/step, {value:.3e} points/s")

    # roofline of the dominant kernel (fused kernel summation)
    ksum_ms = sum(s["ms_sketch_kernel"] for s in stats)
    ksum_n = sum(s["sketch_launches"] for s in stats)
    ksum_flops = sum(s["sketch_flops"] for s in stats)
    ksum_pairs = sum(s["sketch_pairs"] for s in stats)
    if prec == "mixed":
        # entries generated per second against the special-function-unit bound
        achieved = ksum_pairs / (ksum_ms * 1e-3) / 1e9 if ksum_ms > 0 else None
        peak, r_unit = SFU_PEAK_GPAIRS, "Gpair/s"
    else:
        achieved = ksum_flops / (ksum_ms * 1e-3) / 1e12 if ksum_ms > 0 else None
        peak, r_unit = FP64_PEAK_TFLOPS, "TFLOP/s"
    ksum_tflops = ksum_flops / (ksum_ms * 1e-3) / 1e12 if ksum_ms > 0 else None
    phases = {p: statistics.mean(s[f"ms_{p}"] for s in stats)
              for p in ("sketch", "nearfield", "qr", "id", "upsweep", "coupling", "bsr", "total")}
    last = stats[-1]

    result = None
    untuned = None
    if rank == 0 and tuned is not None:
        base = {"d0": w.d0, "d_inc": w.d_inc, "prec": prec}
        step(500, prec, schedule=base)
        tb = []
        for k in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step(600 + k, prec, schedule=base)
            e1.record()
            torch.cuda.synchronize()
            tb.append(e0.elapsed_time(e1))
        untuned = dict(base, ms_per_step=statistics.mean(tb),
                       value=w.n / (statistics.mean(tb) / 1e3))
    if rank == 0:
        # accuracy: ||(A_H2 - A) G|| / ||A G|| with A G by FP64 direct summation
        _, h = step(7, prec, timing=False)
        G = torch.from_numpy(W.gaussian_probe(w.n, 8, 3)).to(dev)
        AG = api.ksum_sketch(X, w.kernel, w.params, G, prec="fp64")
        HG = h.matvec(G)
        err_mixed = float(torch.linalg.norm(HG - AG) / torch.linalg.norm(AG))
        del h
        fp64 = None
        if args.fp64_steps > 0:
            step(2000, "fp64")
            t64 = []
            for k in range(args.fp64_steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                _, h64 = step(3000 + k, "fp64")
                e1.record()
                torch.cuda.synchronize()
                t64.append(e0.elapsed_time(e1))
            s64 = h64.stats()
            err64 = float(torch.linalg.norm(h64.matvec(G) - AG) / torch.linalg.norm(AG))
            fp64 = {"value": w.n / (statistics.mean(t64) / 1e3), "unit": "points/s",
                    "ms_per_step": statistics.mean(t64), "steps": len(t64), "warmup": 1,
                    "rel_error": err64, "d_final": s64["d_final"],
                    "rank_range": [s64["rank_min"], s64["rank_max"]],
                    "sketch_kernel_tflops": (s64["sketch_flops"] / (s64["ms_sketch_kernel"] * 1e-3)
                                             / 1e12 if s64["ms_sketch_kernel"] > 0 else None),
                    "sketch_kernel_peak_tflops": FP64_PEAK_TFLOPS}
            del h64

        # end to end through the C ABI with host buffers
        Xh = torch.from_numpy(w.points()).pin_memory()
        e2e_t = []
        for k in range(max(2, min(args.steps, 5))):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Xd = Xh.to(dev, non_blocking=True)
            tree = api.ClusterTree(Xd, w.leaf_size, w.eta)
            h = api.H2Matrix.build(tree, w.kernel, w.params, w.tol, prec=sched["prec"], seed=k,
                                   sketch="ksum", d0=sched["d0"], d_inc=sched["d_inc"],
                                   d_max=w.d_max)
            ranks, skel, _, _ = h.export_level(1)       # device -> host read of the result
            e1.record()
            torch.cuda.synchronize()
            e2e_t.append(e0.elapsed_time(e1))
            del h, tree
        e2e_ms = statistics.mean(e2e_t)
        bi = Xh.numel() * 8
        bo = int(ranks.nbytes + skel.nbytes)

        traffic = profiled_traffic(prec)
        result = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "prec": prec, "schedule": sched,
                       "omega": "Philox4x32-10 on device",
                       "l2": "flushed between timed steps (512 MiB write)",
                       "step": "tree + lists + H2 build, device-resident points"},
            "roofline": {"kernel": ("k_ksum_tc (fused kernel summation: entries generated on "
                                    "the CUDA cores and special-function units, contracted on "
                                    "tcgen05 with two-part FP16 operands)")
                         if sched["prec"] == "mixed" else
                         ("k_ksum32 (fused kernel summation, FP32 CUDA cores)"
                          if sched["prec"] == "mixed_simt" else
                          "k_ksum64 (fused kernel summation, FP64)"),
                         "bound": "alu", "achieved": achieved, "peak": peak, "unit": r_unit,
                         "frac": achieved / peak if achieved else None,
                         "traffic": traffic,
                         "peak_source": ("152 SMs x 16 SFU lanes x 2070 MHz / 2 SFU operations per "
                                         "Matern entry (unit counts and max clock)"
                                         if prec == "mixed" else "nominal GB300 FP64 1.25 TFLOP/s"),
                         "algorithmic_tflops": ksum_tflops,
                         "flops_per_pair": "2*columns + 10", "launches": ksum_n,
                         "avg_launch_ms": ksum_ms / ksum_n if ksum_n else None},
            "cpu_baseline": cpu,
            "e2e": {"value": w.n / (e2e_ms / 1e3), "unit": "points/s",
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "clocks": clk,
            "rel_error": err_mixed,
            "tol": w.tol,
            "fp64": fp64,
            "autotune": tuned,
            "untuned_schedule": untuned,
            "phases_ms": phases,
            "d_final": last["d_final"], "rounds": last["rounds"],
            "rank_range": [last["rank_min"], last["rank_max"]],
            "memory_bytes": last["bytes_dense"] + last["bytes_coupling"] + last["bytes_basis"],
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


# ---------------------------------------------------------------- reference arm
def main_reference(args):
    """The CPU oracle timed on the host cores on a bounded sample of the same
    workload, scaled to the full point count (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from paper_2506_16759_gb300 import workloads as W
    n_full = W.config("c2").n
    for _ in range(args.warmup):
        run_oracle_child(args.ref_sample)
    secs = []
    last = None
    for _ in range(args.steps):
        last = run_oracle_child(args.ref_sample)
        secs.append(scaled_oracle_rate(last, n_full)[1])
    mean = statistics.mean(secs)
    value = n_full / mean
    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD_DESC, "prec": "fp64"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": (f"each step a full oracle build at N={last['n']} of the same "
                                    "workload, scaled to N=131072 as sketch*(N/n)^2 + "
                                    "rest*(N/n); 1 thread")},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main_kernel_only(args):
    """Small processes for ncu captures.  "ksum": only the fused sketch of the
    benchmark workload (N=131072, 32 columns, all points, same launch plan as
    inside a build).  "build": whole builds of the same workload family at
    --n points with the 80/+16 mixed schedule (its first k_ksum_tc launch is
    the 80-column far-only sketch)."""
    import torch

    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import workloads as W
    dev = torch.device("cuda:0")
    w = W.config("c2")
    if args.kernel_only == "paper":
        main_paper_problem(args, dev)
        return
    if args.kernel_only == "build":
        w = W.scaled(w, args.n or w.n)
        X = torch.from_numpy(w.points()).to(dev)
        times = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = api.ClusterTree(X, w.leaf_size, w.eta)
            h = api.H2Matrix.build(tree, w.kernel, w.params, w.tol, prec="mixed", seed=k,
                                   sketch="ksum", d0=80, d_inc=16, d_max=w.d_max)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append((time.perf_counter() - t0) * 1e3)
            st = h.stats()
            del h, tree
        print(json.dumps({"kernel_only": "build", "n": w.n, "ms": statistics.mean(times),
                          "d_final": st["d_final"], "rank_max": st["rank_max"]}), flush=True)
        return
    X = torch.from_numpy(w.points()).to(dev)
    om = torch.from_numpy(w.omega(32)).to(dev)
    times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        api.ksum_sketch(X, w.kernel, w.params, om, prec=args.prec)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
    flops = float(w.n) * w.n * (2 * 32 + 10)
    ms = statistics.mean(times)
    print(json.dumps({"kernel_only": "ksum", "prec": args.prec, "n": w.n, "columns": 32,
                      "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}), flush=True)


def main_paper_problem(args, dev):
    """A Sec. V-A problem sketched through the matvec of an H2 matrix prebuilt
    for its kernel (untimed).  exp3d / helmholtz: timed tree + construction
    with direct entry evaluation, as in the paper.  update: that H2 matrix
    plus a symmetric rank-32 product recompressed into one H2 matrix (entries
    from the operand's representation plus the product's; the operands share
    the tree, so only the construction is timed)."""
    import numpy as np
    import torch

    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import workloads as W
    w = W.paper_problem(args.problem, args.n or 262144)
    X = torch.from_numpy(w.points()).to(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    tree = api.ClusterTree(X, w.leaf_size, w.eta)
    # the operand: an H2 matrix of the kernel (for "update", of the covariance
    # kernel, to which the low-rank product is added)
    kop, pop = (w.extra["operands"][0] if w.kernel == W.K_H2SUM else (w.kernel, w.params))
    lowrank, kw = None, {}
    if "rank" in w.extra:
        U, V = W.low_rank_factors(w.n, w.extra["rank"], w.extra["lowrank_seed"],
                                  w.extra["lowrank_scale"])
        lowrank = (torch.from_numpy(U).to(dev), torch.from_numpy(V).to(dev))
        kw["lowrank"] = lowrank
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pre = api.H2Matrix.build(tree, kop, pop, w.extra["operand_tol"], prec=args.prec, seed=1,
                             sketch="ksum")
    torch.cuda.synchronize()
    pre_ms = (time.perf_counter() - t0) * 1e3

    def step(seed, timing=False):
        tr = api.ClusterTree(X, w.leaf_size, w.eta) if w.kernel != W.K_H2SUM else tree
        return tr, api.H2Matrix.build(tr, w.kernel, w.params, w.tol, prec=args.prec, seed=seed,
                                      sketch="h2sum", operands=[pre], timing=timing,
                                      d0=w.d0, d_inc=w.d_inc, d_max=w.d_max, **kw)

    times = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        tr, h = step(100 + k)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
        del h, tr
    tr, h = step(7, timing=True)
    st = h.stats()
    G = torch.from_numpy(W.gaussian_probe(w.n, 8, 0)).to(dev)
    kernel_part = api.ksum_sketch(X, kop, pop, G, prec="fp64")
    exact = kernel_part if lowrank is None else kernel_part + lowrank[0] @ (lowrank[1].T @ G)
    err = float(torch.linalg.norm(h.matvec(G) - exact) / torch.linalg.norm(exact))
    err_pre = float(torch.linalg.norm(pre.matvec(G) - kernel_part) /
                    torch.linalg.norm(kernel_part))
    ms = statistics.mean(times)
    print(json.dumps({
        "kernel_only": "paper", "problem": w.name, "n": w.n, "prec": args.prec,
        "ms": ms, "points_per_s": w.n / (ms * 1e-3), "steps": args.steps, "warmup": args.warmup,
        "rel_error": err, "operand_rel_error": err_pre, "operand_tol": w.extra["operand_tol"],
        "operand_build_ms": pre_ms, "operand_rank_max": pre.stats()["rank_max"],
        "tol": w.tol, "d_final": st["d_final"],
        "rank_max": st["rank_max"], "rounds": st["rounds"],
        "memory_gb": (st["bytes_dense"] + st["bytes_coupling"] + st["bytes_basis"]) / 1e9,
        "phases_ms": {p: st[f"ms_{p}"] for p in ("sketch", "nearfield", "qr", "id", "upsweep",
                                                 "coupling", "bsr", "total")}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=8192)
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the workload's 32/+16 sample schedule instead of the tuned one")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--kernel-only", default="", choices=["", "ksum", "build", "paper"],
                    help="time only the fused sketch, builds at --n points (for profiling), "
                         "or a paper kernel problem with the H2-matvec sampler")
    ap.add_argument("--problem", default="helmholtz", choices=["exp3d", "helmholtz", "update"],
                    help="kernel problem for --kernel-only paper")
    ap.add_argument("--n", type=int, default=0, help="point count for --kernel-only build")
    args = ap.parse_args()
    if args.kernel_only:
        main_kernel_only(args)
        return
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample)))
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_gpu(args)


if __name__ == "__main__":
    main()
