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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2 build time & points/s at tol, mixed vs FP64 on 1 GB300; % HBM/compute roofline"
WORKLOAD_DESC = ("c2: N=131072 uniform [0,1]^3, Matern-3/2 l=0.1 + 1e-4 nugget, leaf 64, "
                 "eta 0.7, tol 1e-6, adaptive sampling up to 256 columns (schedule in the line's schedule key), "
                 "fused kernel-summation sketch")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- CPU oracle leg
# The oracle's build of the benchmark workload takes minutes on one core, so
# it is timed on a bounded sample of that workload:
#  * the sketch (most of the oracle's time): its direct kernel sums for a
#    seeded sample of rows of the full 131072-point problem, over the column
#    blocks of the oracle's sample schedule; every row costs the same, so the
#    full sketch takes (N / rows) times as long;
#  * the rest (tree, lists, near field, QR tests, IDs, couplings): full oracle
#    builds of the same workload family at three smaller N (sketch excluded,
#    the samples from the dense matrix), fitted as a*N^b and evaluated at N.
# The sketch rows run once on one core and once spread over all host cores
# (spawned worker processes, as the paper's OpenMP code spreads the sketch).
FIT_SIZES = (4096, 8192, 16384)
# Columns the construction of the full 131072-point workload samples with the
# 32/+16 schedule: the first 32 and three rounds of 16, as its FP64 build (the
# oracle's arithmetic, rank for rank) reports; smaller members of the family
# stop earlier, so the sketch sample takes the full size's column blocks.
FULL_D_FINAL = 80
# launch-shape build options the autotuner picks (passed through to every build)
SHAPE_KEYS = ("bsr_engine", "tc_cols", "ksum_split", "queue_order", "sum_engine")
_W_STATE = {}


def _worker_init(cmax):
    from paper_2506_16759_gb300 import workloads as W
    w = W.config("c2")
    _W_STATE["X"] = w.points()
    _W_STATE["om"] = w.omega(cmax)
    _W_STATE["w"] = w


def _worker_rows(task):
    from oracle import h2_oracle as O
    rows, blocks = task
    X, om, w = _W_STATE["X"], _W_STATE["om"], _W_STATE["w"]
    t0 = time.perf_counter()
    for c0, c1 in blocks:
        O.ksum_rows(X, w.kernel, w.params, np.ascontiguousarray(om[:, c0:c1]), rows, chunk=64)
    return time.perf_counter() - t0


def construction_fit(sizes=FIT_SIZES) -> dict:
    """Oracle builds of the benchmark family at `sizes` (sketch excluded)."""
    from oracle import h2_oracle as O
    from paper_2506_16759_gb300 import workloads as W
    pts = []
    for n in sizes:
        w = W.scaled(W.config("c2"), n)
        X = w.points()
        t0 = time.perf_counter()
        t = O.build_cluster_tree(X, w.leaf_size)
        lists = O.dual_traversal(t, w.eta)
        t_tree = time.perf_counter() - t0
        A = O.dense_matrix(X, w.kernel, w.params)
        h = O.build_h2(t, lists, w.kernel, w.params, w.tol, w.omega(), O.dense_sampler(A),
                       w.d0, w.d_inc, w.d_max)
        del A
        pts.append({"n": n, "s": t_tree + h.timings["construct_s"], "d_final": h.d_final})
    ln = np.log([p["n"] for p in pts])
    lt = np.log([p["s"] for p in pts])
    b, a = np.polyfit(ln, lt, 1)
    resid = float(np.max(np.abs(lt - (a + b * ln))))
    return {"points": pts, "exponent": float(b), "log_coef": float(a),
            "max_log_residual": resid, "d_final": pts[-1]["d_final"]}


def sketch_blocks(d_final, d0=32, d_inc=16):
    return [(0, d0)] + [(c, c + d_inc) for c in range(d0, d_final, d_inc)]


def sketch_sample(rows_n, d_final, pool=None, workers=1, seed=0) -> dict:
    """Seconds for the oracle's sketch of `rows_n` sampled rows of the full
    workload (serially, or split over `workers` pool processes)."""
    from paper_2506_16759_gb300 import workloads as W
    n = W.config("c2").n
    rows = np.sort(np.random.default_rng(seed).choice(n, rows_n, replace=False))
    blocks = sketch_blocks(d_final)
    if pool is None:
        _worker_init(blocks[-1][1])
        t = _worker_rows((rows, blocks))
    else:
        parts = np.array_split(rows, workers)
        t0 = time.perf_counter()
        pool.map(_worker_rows, [(p, blocks) for p in parts])
        t = time.perf_counter() - t0
    return {"rows": rows_n, "s": t, "full_s": t * n / rows_n, "blocks": len(blocks),
            "columns": blocks[-1][1]}


def make_pool(d_final):
    import multiprocessing as mp
    workers = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    return ctx.Pool(workers, initializer=_worker_init, initargs=(sketch_blocks(d_final)[-1][1],)), \
        workers


def oracle_baseline(rows_serial: int, rows_parallel: int) -> dict:
    """The CPU oracle's rate on the benchmark workload (runs in a child
    process with single-threaded BLAS)."""
    from paper_2506_16759_gb300 import workloads as W
    n = W.config("c2").n
    fit = construction_fit()
    rest = math.exp(fit["log_coef"]) * n ** fit["exponent"]
    ser = sketch_sample(rows_serial, FULL_D_FINAL)
    pool, workers = make_pool(FULL_D_FINAL)
    with pool:
        pool.map(_worker_rows, [(np.arange(1), [(0, 1)])] * workers)   # workers loaded
        par = sketch_sample(rows_parallel, FULL_D_FINAL, pool, workers)
    return {"n": n, "fit": fit, "rest_s": rest, "serial": ser, "parallel": par,
            "workers": workers,
            "secs_1": ser["full_s"] + rest, "secs_p": par["full_s"] + rest}


def run_oracle_child(*args) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), *args],
                         capture_output=True, text=True, env=env, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def describe_baseline(r: dict) -> str:
    f = r["fit"]
    pts = ", ".join(f"N={p['n']}: {p['s']:.2f}s" for p in f["points"])
    return (f"sketch: the oracle's direct kernel sums for {r['parallel']['rows']} seeded rows of "
            f"the full N={r['n']} problem over its {r['parallel']['blocks']} column blocks "
            f"({r['parallel']['columns']} columns) on {r['workers']} processes "
            f"({r['parallel']['s']:.2f}s; one core, {r['serial']['rows']} rows: "
            f"{r['serial']['s']:.2f}s), scaled by N/rows; the rest of the build: oracle builds "
            f"at {pts} (sketch excluded), fitted as a*N^b with b={f['exponent']:.3f} "
            f"(max log residual {f['max_log_residual']:.3f}) -> {r['rest_s']:.1f}s at N; "
            f"estimated build {r['secs_p']:.0f}s on {r['workers']} cores, "
            f"{r['secs_1']:.0f}s on one")


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
    # the sources the tensor-core sketch kernel is compiled from
    for f in ("sketch_tc.cu", "tc_ptx.cuh", "h2_internal.cuh", "h2_types.h", "h2_ops.h"):
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
PEAK_NAMES = ("fp64_tflops", "fp32_tflops", "sfu_ex2_gops", "f16_tc_tflops", "tf32_tc_tflops",
              "sfu_sqrt_gops", "sfu_rsqrt_gops")


def measure_peaks() -> dict:
    """Measured pipe throughputs of this device (h2_measure_peak) plus the
    measured HBM copy bandwidth and cuBLAS BF16 rate."""
    import ctypes
    import torch
    from paper_2506_16759_gb300 import _lib
    L = _lib.lib()
    out = {}
    for w, name in enumerate(PEAK_NAMES):
        v = ctypes.c_double()
        st = L.h2_measure_peak(w, torch.cuda.current_stream().cuda_stream, ctypes.byref(v))
        out[name] = v.value if st == 0 else None
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        d = json.load(open(mp))
        out["hbm_gbs"] = d.get("hbm_gbs")
        out["bf16_tflops"] = d.get("bf16_tflops")
        out["hbm_source"] = "MEASURED_PEAKS.json (STREAM-style copy)"
    else:
        out["hbm_gbs"], out["bf16_tflops"] = 6800.0, 1900.0
        out["hbm_source"] = "fallback (no MEASURED_PEAKS.json)"
    return out


# Special-function operations per kernel entry in the tensor-core sketch:
# square root and exp2 (exponential, Matern), exp2 (Gaussian), reciprocal
# square root (Laplace, Helmholtz; its cosine is a polynomial).
SFU_OPS = {0: ("sqrt", "ex2"), 1: ("sqrt", "ex2"), 2: ("ex2",), 3: ("rsqrt",), 6: ("rsqrt",)}


def sfu_pair_peak(kid: int, peaks: dict):
    """Entries per second (G) the special-function units allow: they share one
    pipe, so the times of an entry's operations add."""
    ops = SFU_OPS.get(kid)
    if not ops or any(not peaks.get(f"sfu_{o}_gops") for o in ops):
        return None, None
    per = sum(1.0 / peaks[f"sfu_{o}_gops"] for o in ops)
    src = " + ".join(f"1/{peaks[f'sfu_{o}_gops']:.0f} ({o})" for o in ops)
    return 1.0 / per, f"1 / ({src}) G entries/s from the measured rates (h2_measure_peak)"


def sketch_roofline(stats: list, kid: int, prec: str, peaks: dict, timed_alone: bool) -> dict:
    """Roofline of the fused sketch over the launches of instrumented builds:
    entries per second against the special-function-unit bound (mixed), or
    FP64 flops against the measured FP64 FMA rate."""
    ms = sum(s["ms_sketch_kernel"] for s in stats)
    n = sum(s["sketch_launches"] for s in stats)
    pairs = sum(s["sketch_pairs"] for s in stats)
    flops = sum(s["sketch_flops"] for s in stats)
    if ms <= 0:
        return None
    peak, src = sfu_pair_peak(kid, peaks)
    if prec == "mixed" and peak:
        achieved = pairs / (ms * 1e-3) / 1e9
        return {"kernel": "k_ksum_tc (fused kernel summation: entries on the CUDA cores and "
                          "special-function units, contracted on tcgen05 with two-part operands)",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": achieved / peak, "peak_source": src,
                "algorithmic_tflops": flops / (ms * 1e-3) / 1e12, "launches": n,
                "avg_launch_ms": ms / n if n else None}
    achieved = flops / (ms * 1e-3) / 1e12
    peak = peaks.get("fp64_tflops") if prec == "fp64" else peaks.get("fp32_tflops")
    return {"kernel": "k_ksum64 (fused kernel summation, FP64)" if prec == "fp64" else
            "k_ksum32 (fused kernel summation, FP32 CUDA cores)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None,
            "peak_source": "measured FMA rate (h2_measure_peak)",
            "flops_per_pair": "2*columns + 10", "launches": n,
            "avg_launch_ms": ms / n if n else None}


def timed(fn, steps, flush):
    """CUDA-event milliseconds of `steps` calls of fn() (L2 flushed before each)."""
    import torch
    out = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def extra_configs(dev, flush, peaks, names, fp64_steps) -> dict:
    """The other workloads: mixed and FP64 build times, points/s, errors and
    the roofline of each one's dominant kernel."""
    import torch
    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import workloads as W
    res = {}

    def probe_err(h, X, kid, params, n):
        G = torch.from_numpy(W.gaussian_probe(n, 8, 3)).to(dev)
        AG = api.ksum_sketch(X, kid, params, G, prec="fp64")
        return float(torch.linalg.norm(h.matvec(G) - AG) / torch.linalg.norm(AG))

    def run_single(name, w, sched, extra_kw=None, err_fn=None, roof_fn=None, tree=None):
        X = torch.from_numpy(w.points()).to(dev)
        kw = dict(extra_kw or {})
        entry = {"n": w.n, "tol": w.tol}
        for prec in ("mixed", "fp64"):
            sc = sched if prec == "mixed" else {"d0": w.d0, "d_inc": w.d_inc}
            holder = {}

            def build(timing=False, seed=0):
                tr = tree if tree is not None else api.ClusterTree(X, w.leaf_size, w.eta)
                holder["h"] = api.H2Matrix.build(tr, w.kernel, w.params, w.tol, prec=prec,
                                                 seed=seed, sketch=w.sketch, timing=timing,
                                                 d0=sc["d0"], d_inc=sc["d_inc"], d_max=w.d_max,
                                                 **kw)
                holder["t"] = tr
            steps = 3 if prec == "mixed" else fp64_steps
            if steps <= 0:
                continue
            build(seed=90)
            ms = statistics.mean(timed(lambda: build(seed=91), steps, flush))
            flush.zero_()
            build(timing=True, seed=92)
            st = holder["h"].stats()
            e = {"ms_per_build": ms, "points_per_s": w.n / (ms * 1e-3), "steps": steps,
                 "schedule": sc, "d_final": st["d_final"], "rounds": st["rounds"],
                 "rank_range": [st["rank_min"], st["rank_max"]],
                 "memory_bytes": st["bytes_dense"] + st["bytes_coupling"] + st["bytes_basis"],
                 "phases_ms": {p: st[f"ms_{p}"] for p in ("sketch", "nearfield", "qr", "id",
                                                         "upsweep", "coupling", "bsr")}}
            e["rel_error"] = err_fn(holder["h"], X) if err_fn else None
            e["roofline"] = roof_fn(st, prec) if roof_fn else None
            entry[prec] = e
            holder.clear()
        res[name] = entry

    if "c1" in names:
        w = W.config("c1")
        Xh = w.points()
        from oracle import h2_oracle as O   # noqa: F401  (not used: A comes from the library)
        X = torch.from_numpy(Xh).to(dev)
        idx = torch.arange(w.n, dtype=torch.int32, device=dev)
        A = api.entry_block(X, w.kernel, w.params, idx, idx)

        def dense_roof(st, prec):
            cols = st["sketch_columns"]
            flops = 2.0 * w.n * w.n * cols
            ms = st["ms_sketch"]
            pk = peaks.get("fp64_tflops")
            a = flops / (ms * 1e-3) / 1e12 if ms > 0 else None
            return {"kernel": "k_dense_gemm64 (dense sketch Y = A Omega, FP64)", "bound": "alu",
                    "achieved": a, "peak": pk, "unit": "TFLOP/s",
                    "frac": a / pk if a and pk else None,
                    "note": "sketch phase time (includes the permutations of Omega and Y)"}

        def dense_err(h, _X):
            G = torch.from_numpy(W.gaussian_probe(w.n, 8, 3)).to(dev)
            AG = A @ G
            return float(torch.linalg.norm(h.matvec(G) - AG) / torch.linalg.norm(AG))
        run_single("c1", w, {"d0": w.d0, "d_inc": w.d_inc}, {"dense_a": A}, dense_err,
                   dense_roof)
        del A
    if "c3" in names:
        w = W.config("c3")

        def c3_roof(st, prec):
            return sketch_roofline([st], w.kernel, prec, peaks, False)
        run_single("c3", w, {"d0": 64, "d_inc": 32}, None,
                   lambda h, X: probe_err(h, X, w.kernel, w.params, w.n), c3_roof)
    if "c5" in names:
        insts = W.c5_instances()
        Xs = [torch.from_numpy(i.points()).to(dev) for i in insts]
        ntot = sum(i.n for i in insts)
        entry = {"instances": len(insts), "n_total": ntot, "tol": 1e-6}
        for prec in ("mixed", "fp64"):
            holder = {}
            steps = 3 if prec == "mixed" else fp64_steps
            if steps <= 0:
                continue

            def build(timing=False, seed=0):
                trees = [api.ClusterTree(X, i.leaf_size, i.eta) for X, i in zip(Xs, insts)]
                holder["h"] = api.H2Matrix.build_batched(
                    trees, [i.kernel for i in insts], [i.params for i in insts],
                    [i.tol for i in insts], prec=prec, seed=seed, timing=timing)
            build(seed=80)
            ms = statistics.mean(timed(lambda: build(seed=81), steps, flush))
            flush.zero_()
            build(timing=True, seed=82)
            st = holder["h"].stats()
            G = torch.from_numpy(W.gaussian_probe(ntot, 8, 3)).to(dev)
            y = holder["h"].matvec(G)
            errs, off = [], 0
            for X, i in zip(Xs, insts):
                AG = api.ksum_sketch(X, i.kernel, i.params, G[off:off + i.n], prec="fp64")
                errs.append(float(torch.linalg.norm(y[off:off + i.n] - AG) / torch.linalg.norm(AG)))
                off += i.n
            entry[prec] = {"ms_per_build": ms, "points_per_s": ntot / (ms * 1e-3),
                           "steps": steps, "max_rel_error": max(errs),
                           "d_final": st["d_final"], "rank_range": [st["rank_min"], st["rank_max"]],
                           "kernel_launches": st["kernel_launches"],
                           "roofline": sketch_roofline([st], 0, prec, peaks, False),
                           "step": "64 trees + one batched build (leaf 64, 32/+16 samples)"}
            holder.clear()
        res["c5"] = entry
    if "c4" in names:
        w = W.config("c4")
        X = torch.from_numpy(w.points()).to(dev)
        tree = api.ClusterTree(X, w.leaf_size, w.eta)
        t0 = time.perf_counter()
        ops = [api.H2Matrix.build(tree, k, p, w.extra["operand_tol"], prec="mixed", seed=3 + q)
               for q, (k, p) in enumerate(w.extra["operands"])]
        torch.cuda.synchronize()
        op_s = time.perf_counter() - t0
        op_bytes = 0
        for o in ops:
            so = o.stats()
            op_bytes += so["bytes_dense"] + so["bytes_coupling"] + so["bytes_basis"]

        def c4_err(h, _X):
            G = torch.from_numpy(W.gaussian_probe(w.n, 8, 3)).to(dev)
            AG = ops[0].matvec(G) + ops[1].matvec(G)
            return float(torch.linalg.norm(h.matvec(G) - AG) / torch.linalg.norm(AG))

        def c4_roof(st, prec):
            calls = 1 + st["rounds"]
            ms = st["ms_sketch"]
            cols = st["sketch_columns"]
            byts = op_bytes * calls + 2.0 * w.n * cols * 8 * len(ops)
            a = byts / (ms * 1e-3) / 1e9 if ms > 0 else None
            pk = peaks.get("hbm_gbs")
            return {"kernel": "operand H2 matvecs (k_bsr_* block-sparse products, k_basis_* "
                              "basis products)", "bound": "hbm", "achieved": a, "peak": pk,
                    "unit": "GB/s", "frac": a / pk if a and pk else None,
                    "traffic": None,
                    "algorithmic_bytes": "operand blocks (D, B, U/E) once per sketch call + "
                                         "x and y panels in FP64",
                    "note": "sketch phase time: every operand matvec of the build"}
        # mixed builds take the tensor-core couplings (sum_engine 1)
        run_single("c4", w, {"d0": 80, "d_inc": 16}, {"operands": ops, "sum_engine": 1}, c4_err,
                   c4_roof, tree=tree)
        res["c4"]["operands"] = {"tol": w.extra["operand_tol"], "prec": "mixed",
                                 "build_s": op_s, "bytes": op_bytes}
        del ops
    return res


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
            r = run_oracle_child("--oracle-baseline", str(args.cpu_rows), str(args.cpu_rows_par))
            n = r["n"]
            cpu = {"value": n / r["secs_p"], "unit": "points/s", "cores": r["workers"],
                   "kind": "oracle", "sample": describe_baseline(r),
                   "single_core": {"value": n / r["secs_1"], "unit": "points/s", "cores": 1}}
        except Exception as e:  # the baseline must not sink the GPU line
            cpu = {"value": None, "unit": "points/s", "cores": None, "kind": "oracle",
                   "sample": f"failed: {e}"}

    peaks = measure_peaks() if rank == 0 else {}
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
        sched = {k: kw[k] for k in ("d0", "d_inc", "prec", "bsr_engine", "tc_cols",
                                    "ksum_split", "queue_order")}
        tuned = dict(sched, tuning_s=time.perf_counter() - t0, build_ms=ms)
        log(f"[bench] autotuned schedule {sched} ({ms:.1f} ms build)")

    def step(seed, precision, timing=True, schedule=None):
        sc = schedule or sched
        if precision == "fp64":
            sc = {"d0": w.d0, "d_inc": w.d_inc, "prec": "fp64"}
        tree = api.ClusterTree(X, w.leaf_size, w.eta)
        shapes = {k: sc[k] for k in SHAPE_KEYS if k in sc}
        h = api.H2Matrix.build(tree, w.kernel, w.params, w.tol, prec=sc["prec"], seed=seed,
                               sketch="ksum", timing=timing, d0=sc["d0"], d_inc=sc["d_inc"],
                               d_max=w.d_max, **shapes)
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

    phases = {p: statistics.mean(s[f"ms_{p}"] for s in stats)
              for p in ("sketch", "nearfield", "qr", "id", "upsweep", "coupling", "bsr", "total")}
    last = stats[-1]

    result = None
    untuned = None
    if rank == 0 and tuned is not None:
        base = {"d0": w.d0, "d_inc": w.d_inc, "prec": prec}
        step(500, prec, schedule=base)
        tb = timed(lambda: step(600, prec, schedule=base), 3, flush)
        untuned = dict(base, ms_per_step=statistics.mean(tb),
                       value=w.n / (statistics.mean(tb) / 1e3))
    if rank == 0:
        roof = sketch_roofline(stats, w.kernel, sched["prec"], peaks, False)
        if roof is not None:
            roof["traffic"] = profiled_traffic(prec)
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
            holder = {}

            def run64():
                holder["h"] = step(3000, "fp64")[1]
            t64 = timed(run64, args.fp64_steps, flush)
            h64 = holder["h"]
            s64 = h64.stats()
            err64 = float(torch.linalg.norm(h64.matvec(G) - AG) / torch.linalg.norm(AG))
            flush.zero_()
            _, h64t = step(3100, "fp64", timing=True)
            fp64 = {"value": w.n / (statistics.mean(t64) / 1e3), "unit": "points/s",
                    "ms_per_step": statistics.mean(t64), "steps": len(t64), "warmup": 1,
                    "rel_error": err64, "d_final": s64["d_final"],
                    "rank_range": [s64["rank_min"], s64["rank_max"]],
                    "roofline": sketch_roofline([h64t.stats()], w.kernel, "fp64", peaks, False)}
            del h64, h64t
            holder.clear()

        # end to end through the C ABI with host buffers: points in, the
        # level-1 ranks and skeletons out (the H2 matrix itself stays on the
        # device, where its matvec is used)
        Xh = torch.from_numpy(w.points()).pin_memory()
        e2e_t = []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Xd = Xh.to(dev, non_blocking=True)
            tree = api.ClusterTree(Xd, w.leaf_size, w.eta)
            h = api.H2Matrix.build(tree, w.kernel, w.params, w.tol, prec=sched["prec"], seed=k,
                                   sketch="ksum", d0=sched["d0"], d_inc=sched["d_inc"],
                                   d_max=w.d_max,
                                   **{k2: sched[k2] for k2 in SHAPE_KEYS if k2 in sched})
            ranks, skel, _, _ = h.export_level(1)       # device -> host read of the result
            e1.record()
            torch.cuda.synchronize()
            e2e_t.append(e0.elapsed_time(e1))
            del h, tree
        e2e_ms = statistics.mean(e2e_t)
        bi = Xh.numel() * 8
        bo = int(ranks.nbytes + skel.nbytes)

        extras = {}
        if args.configs:
            names = [c for c in args.configs.split(",") if c]
            log(f"[bench] other workloads: {names}")
            extras = extra_configs(dev, flush, peaks, names, args.fp64_steps)

        result = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
            "config": bench_config(),
            "prec": prec, "schedule": sched,
            "roofline": roof,
            "peaks": peaks,
            "cpu_baseline": cpu,
            "e2e": {"value": w.n / (e2e_ms / 1e3), "unit": "points/s",
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms,
                    "steps": len(e2e_t),
                    "result": "level-1 ranks and skeleton indices read back; the H2 matrix "
                              "stays on the device"},
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
            "configs": extras,
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def bench_config() -> dict:
    """The workload every arm of the benchmark measures (identical keys)."""
    return {"workload": WORKLOAD_DESC,
            "l2": "flushed between timed steps (512 MiB write)",
            "step": "tree + lists + H2 build from device-resident points"}


# ---------------------------------------------------------------- reference arm
def main_reference(args):
    """The CPU oracle on the host cores (rank 0 only).  Each step times the
    oracle's sketch of sampled rows of the full workload on all cores and an
    oracle build of the same family at N=8192 (sketch excluded), and scales
    them to the full build: rows by N/rows, the build by (N/8192)^b with b
    fitted in the warm-up from builds at three sizes."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    r = run_oracle_child("--oracle-reference", str(args.steps), str(max(args.warmup, 0)),
                         str(args.ref_rows))
    value = r["n"] / statistics.mean(r["secs"])
    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(r["wall"]) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": bench_config(), "prec": "fp64",
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": r["workers"],
                         "kind": "oracle",
                         "sample": (f"each step: the oracle's sketch of {args.ref_rows} seeded "
                                    f"rows of the full problem on {r['workers']} processes, "
                                    "scaled by N/rows, plus an oracle build at N=8192 (sketch "
                                    f"excluded) scaled by (N/8192)^{r['exponent']:.3f} (exponent "
                                    "fitted in the warm-up at N=4096/8192/16384); ms_per_step is "
                                    "the measured wall time of one such step, value the "
                                    "estimated rate of the full build")},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_reference_steps(steps: int, warmup: int, rows: int) -> dict:
    """Child process of the reference arm."""
    from paper_2506_16759_gb300 import workloads as W
    n = W.config("c2").n
    fit = construction_fit()
    b = fit["exponent"]
    pool, workers = make_pool(FULL_D_FINAL)
    secs, wall = [], []
    with pool:
        pool.map(_worker_rows, [(np.arange(1), [(0, 1)])] * workers)
        for k in range(max(warmup - 1, 0) + steps):
            t0 = time.perf_counter()
            sk = sketch_sample(rows, FULL_D_FINAL, pool, workers, seed=k)
            c = construction_fit((8192,))
            el = time.perf_counter() - t0
            if k >= max(warmup - 1, 0):
                secs.append(sk["full_s"] + c["points"][0]["s"] * (n / 8192) ** b)
                wall.append(el)
    return {"n": n, "secs": secs, "wall": wall, "workers": workers, "exponent": b}


def main_kernel_only(args):
    """Small processes for ncu captures.  "ksum": only the fused sketch of the
    benchmark workload (N=131072, 32 columns, all points, same launch plan as
    inside a build).  "build": whole builds of the same workload family at
    --n points with the 80/+16 mixed schedule and the work-queue order (the
    tuned choice on this workload; its first k_ksum_tc launch is the
    80-column far-only sketch).  "paper": a Sec. V-A problem.  "matvec": the
    H2 matvec of a 1e-8 operand."""
    import torch

    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import workloads as W
    dev = torch.device("cuda:0")
    w = W.config("c2")
    if args.kernel_only == "paper":
        main_paper_problem(args, dev)
        return
    if args.kernel_only == "matvec":
        main_matvec(args, dev)
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
                                   sketch="ksum", d0=80, d_inc=16, d_max=w.d_max,
                                   bsr_engine=args.bsr_engine, queue_order=1,
                                   timing=args.phases)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append((time.perf_counter() - t0) * 1e3)
            st = h.stats()
            del h, tree
        out = {"kernel_only": "build", "n": w.n, "ms": statistics.mean(times),
               "bsr_engine": args.bsr_engine, "d_final": st["d_final"],
               "rank_max": st["rank_max"]}
        if args.phases:
            out["phases_ms"] = {p: st[f"ms_{p}"] for p in ("sketch", "nearfield", "qr", "id",
                                                         "upsweep", "coupling", "bsr", "total")}
        print(json.dumps(out), flush=True)
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


def main_matvec(args, dev):
    """The H2 matrix-vector product on its own: the first operand of the
    H2-sum workload (exp(-r/0.1) on 2^18 uniform points in [0,1]^3, built in
    mixed precision at tol 1e-8) applied to 16 and 80 Gaussian columns.  The
    product reads every stored block once (near-field D, couplings B, bases
    E), so its roofline is HBM bandwidth over the operand's bytes."""
    import torch

    from paper_2506_16759_gb300 import api
    from paper_2506_16759_gb300 import workloads as W
    w = W.config("c4")
    if args.n:
        w = W.scaled(w, args.n)
    kop, pop = w.extra["operands"][0]
    X = torch.from_numpy(w.points()).to(dev)
    tree = api.ClusterTree(X, w.leaf_size, w.eta)
    op = api.H2Matrix.build(tree, kop, pop, w.extra["operand_tol"], prec="mixed", seed=3)
    st = op.stats()
    op_bytes = st["bytes_dense"] + st["bytes_coupling"] + st["bytes_basis"]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {"kernel_only": "matvec", "n": w.n, "operand_tol": w.extra["operand_tol"],
           "operand_bytes": op_bytes, "rank_max": st["rank_max"], "columns": {}}
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(mp)).get("hbm_gbs") if os.path.exists(mp) else 6800.0
    out["hbm_peak_gbs"] = hbm
    for cols in (16, 80):
        G = torch.from_numpy(W.gaussian_probe(w.n, cols, 0)).to(dev)
        for _ in range(args.warmup):
            op.matvec(G)
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            op.matvec(G)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.mean(times)
        gbs = (op_bytes + 2.0 * w.n * cols * 8) / (ms * 1e-3) / 1e9
        out["columns"][str(cols)] = {"ms": ms, "gb_per_s": gbs,
                                     "hbm_frac": gbs / hbm if hbm else None}
    print(json.dumps(out), flush=True)


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
    ap.add_argument("--cpu-rows", type=int, default=64,
                    help="sketch rows of the one-core oracle sample")
    ap.add_argument("--cpu-rows-par", type=int, default=1024,
                    help="sketch rows of the all-cores oracle sample")
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="sketch rows per step of the reference arm")
    ap.add_argument("--configs", default="c1,c3,c5,c4",
                    help="other workloads reported beside the headline ('' = none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the workload's 32/+16 sample schedule instead of the tuned one")
    ap.add_argument("--oracle-baseline", nargs=2, type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-reference", nargs=3, type=int, default=None,
                    help=argparse.SUPPRESS)
    ap.add_argument("--kernel-only", default="", choices=["", "ksum", "build", "paper", "matvec"],
                    help="time only the fused sketch, builds at --n points (for profiling), "
                         "or a paper kernel problem with the H2-matvec sampler")
    ap.add_argument("--problem", default="helmholtz", choices=["exp3d", "helmholtz", "update"],
                    help="kernel problem for --kernel-only paper")
    ap.add_argument("--n", type=int, default=0, help="point count for --kernel-only build")
    ap.add_argument("--bsr-engine", type=int, default=0, choices=[0, 1],
                    help="--kernel-only build: block-sparse products on tensor cores (0) or "
                         "CUDA cores (1)")
    ap.add_argument("--phases", action="store_true",
                    help="--kernel-only build: per-phase device times (synchronising timers)")
    args = ap.parse_args()
    if args.kernel_only:
        main_kernel_only(args)
        return
    if args.oracle_baseline:
        print(json.dumps(oracle_baseline(*args.oracle_baseline)))
        return
    if args.oracle_reference:
        print(json.dumps(oracle_reference_steps(*args.oracle_reference)))
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_gpu(args)


if __name__ == "__main__":
    main()
