#!/usr/bin/env python3
"""Throughput of batched NTU bond updates on GB300.

One step = one pass of the whole bond update (gate split and QR, exact
eight-site environment metric, Hermitise/repair, SVDU start + ALS sweeps,
recompose) over a batch of independent synthetic bond updates shaped like the
paper's workloads: D=8, d=2, gate exp(-i 0.01 ZZ) split at r=2, iid complex
N(0,1) site tensors (seed 5, normalised), 10 ALS sweeps.  The headline path
is the mixed one (FP32 environment contraction, FP64 solvers); the plain FP64
path is measured on the same GPU for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_06635_gb300 import inputs as I  # noqa: E402

METRIC = "NTU bond updates/s"
FP64_PEAK = 1.25e12          # nominal GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)
FP32_SIMT_PEAK = 152 * 128 * 2 * 2.07e9   # nominal FP32 FMA pipes
# What each precision computes in which arithmetic (the mixed contexts keep
# FP64 for the solves, SVDs and eigendecompositions; the ALS reduced
# metrics, g x0, the final error and the QR's Gram products are double-FP32
# pairs, about 2^-48 relative).
DTYPE_BF16X3 = "split-bf16 env (fp32 acc) + double-fp32 ALS metric build + c128 solves"
DTYPE_FP32 = "c64 env + double-fp32 ALS metric build + c128 solves"
PRECISION_BF16X3 = ("mixed: split-BF16 tcgen05 environment with FP32 accumulation; "
                    "CholeskyQR2, ALS reduced metrics, g x0 and final error in double-FP32 "
                    "(~2^-48); FP64 solves, SVDs and eigendecompositions")
PRECISION_FP32 = ("mixed: FP32 environment; CholeskyQR2, ALS reduced metrics, g x0 and final "
                  "error in double-FP32 (~2^-48); FP64 solves, SVDs and eigendecompositions")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------- algorithmic work
def env_flops(D, r, d_p=2):
    """Real flops of the environment contraction of one bond update:
    8 x complex MACs of edge tensors, half networks and join (Fig. 4)."""
    mac = d_p * (2 * D ** 5 + 4 * D ** 6) + 2 * (d_p * D ** 5 * r + d_p * D ** 7 * r * r
                                                 + 2 * D ** 8 * r * r) + D ** 8 * r ** 4
    return 8.0 * mac


def als_flops(D, r, sweeps):
    """Algorithmic real flops of the ALS stage of one bond update (Fig. 5):
    per sweep the two reduced problems, 2 (K^4 D + K^3 D^2) complex
    multiply-adds (g_A = (1 x M_B)^H g (1 x M_B) and its source, then the
    same for M_B), times 8.  The eigendecompositions of the full count (one
    of g, two of g_A per sweep) are not credited: the certified solves that
    the measured workload takes (Gershgorin discs + conjugate gradients)
    perform none."""
    K = D * r
    return sweeps * 2 * 8.0 * (K ** 4 * D + K ** 3 * D * D)


def als_peak(precision, gemm_peaks):
    """Measured ceiling of the pipe the ALS contraction runs on: on the mixed
    contexts the reduced metrics are built in double-FP32 arithmetic on the
    FP32 lanes, so the in-run FP32 GEMM rate (cuBLAS SGEMM, no TF32); on the
    FP64 context the in-run FP64 GEMM rate.  Nominal unit-count peaks when no
    measurement is available."""
    if precision == "fp64":
        if "fp64_tflops" in gemm_peaks:
            return gemm_peaks["fp64_tflops"] * 1e12, "measured fp64 GEMM (cuBLAS DGEMM, this run)"
        return FP64_PEAK, "nominal FP64 (152 SMs x 2 DFMA/clk x 2 x 2.07 GHz)"
    if "fp32_tflops" in gemm_peaks:
        return gemm_peaks["fp32_tflops"] * 1e12, ("measured fp32 GEMM (cuBLAS SGEMM, no TF32, "
                                                   "this run): the ceiling of the lane build "
                                                   "(double-FP32 on the FP32 lanes); the "
                                                   "tensor-core build emulates the same FP64-"
                                                   "accurate contraction with 21 exact BF16 "
                                                   "slice products, so it is held to the same "
                                                   "ceiling")
    return FP32_SIMT_PEAK, "nominal FP32 lanes (152 x 128 x 2 x 2.07 GHz)"


def als_traffic(precision, D, r, sweeps, items):
    """DRAM bytes of the ALS stage's launches (k_gmax, k_gsplit, k_oz_slice,
    k_als) from the ncu capture recorded in profiles/traffic.json, scaled by
    items (every item's data is private); None when the kernel sources
    changed since the capture or the workload differs."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_als"]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if (h.hexdigest() != rec["sources_sha256"] or rec["precision"] != precision
                or (rec["D"], rec["r"], rec["sweeps"]) != (D, r, sweeps)):
            return None
        return rec["dram_bytes_per_item"] * items
    except Exception:
        return None


def env_roof(precision, achieved, peaks):
    """Environment throughput against the peak of the pipe it runs on: the
    BF16 tensor cores (measured dense peak; the split products issue 3x the
    algorithmic flops), FP32 FMA or FP64."""
    if precision == "bf16x3":
        if "bf16_tflops" in peaks:
            peak, src = peaks["bf16_tflops"] * 1e12, "measured bf16 dense (MEASURED_PEAKS.json)"
        else:
            peak, src = 1900.0e12, "fallback bf16 dense 1.9 PFLOP/s (no measured peak)"
        return {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "issued_frac": 3 * achieved / peak, "peak_source": src}
    key = "fp32_tflops" if precision == "fp32" else "fp64_tflops"
    if key in peaks:
        peak = peaks[key] * 1e12
        src = f"measured {key[:4]} GEMM (cuBLAS via torch.matmul, this run)"
    else:
        peak = FP32_SIMT_PEAK if precision == "fp32" else FP64_PEAK
        src = "nominal from unit counts and clocks"
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src}


def measure_gemm_peaks(n: int = 8192, reps: int = 5) -> dict:
    """FP64 and FP32 (no TF32) GEMM rates of this GPU through the vendor BLAS
    (torch.matmul), in TFLOP/s: the measured ceilings of the FP64 and FP32
    environment paths, taken like the measured BF16 peak."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt in (("fp64_tflops", torch.float64), ("fp32_tflops", torch.float32)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            out[name] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


# ---------------------------------------------------- multi-rank bookkeeping
def reduce_max(x: float, dist=None, device: str = "cpu") -> float:
    """The largest value of x over all ranks (x itself without a process
    group): the step time of the job is that of its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, items_per_rank: int, ms_max: float) -> float:
    """Whole-job throughput: every rank updates its own items_per_rank bonds
    per step (weak scaling) and the step lasts ms_max, the slowest rank's."""
    return world * items_per_rank / (ms_max / 1e3)


def rank_seed(rank: int, base: int = 5) -> int:
    """Seed of a rank's synthetic batch: ranks draw disjoint inputs."""
    return base + 1000 * rank


# ------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl)
                          if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ oracle leg
def _oracle_rate(D, r, sweeps, seconds, seed, max_items=64, threads=None, keep=(),
                 batch=None, tau_kmax=15):
    """Bond updates/s of the CPU oracle on items of the workload, run in a
    fresh child process with `threads` BLAS threads (default: every host
    core).  The items in `keep` (indices into the workload's batch of
    `batch` items) run first and their results -- delta, eps0, the repaired
    metric g, A' and B' -- come back for the accuracy check; the rest are
    the first items of the batch.  Returns (rate, n, seconds, threads,
    kept results)."""
    cores = len(os.sched_getaffinity(0))
    threads = threads or cores
    batch = batch or max_items
    fd, out_path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I
cfg = O.Config(D={D}, r={r}, sweeps={sweeps}, tau_exponents=tuple(range(4, {tau_kmax} + 1)))
keep = {list(keep)!r}
Ta, Tb, G = I.batch_items({seed}, {batch}, 2, {D}, I.zz_gate(0.01))
order = keep + [i for i in range({max_items}) if i not in keep]
O.bond_update(Ta[order[0]], Tb[order[0]], G[order[0]], cfg)     # warm-up (BLAS, caches)
res = {{}}
t0 = time.perf_counter(); n = 0
while n < len(order) and (n < max(2, len(keep)) or time.perf_counter() - t0 < {seconds}):
    i = order[n]
    A2, B2, info = O.bond_update(Ta[i], Tb[i], G[i], cfg, keep=i in keep)
    if i in keep:
        res[f"g{{i}}"] = info.g; res[f"A{{i}}"] = A2; res[f"B{{i}}"] = B2
        res[f"d{{i}}"] = np.array([info.delta, info.eps0])
        res[f"x{{i}}"] = np.array([O.measure(A2, B2, 0, I.pauli("X"), 1).real])
    n += 1
dt = time.perf_counter() - t0
np.savez({out_path!r}, **res)
print(json.dumps({{"n": n, "seconds": dt}}))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             env=env, timeout=900)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        res = json.loads(out.stdout.strip().splitlines()[-1])
        kept = dict(np.load(out_path)) if keep else {}
    finally:
        os.unlink(out_path)
    return res["n"] / res["seconds"], res["n"], res["seconds"], threads, kept


def _oracle_rate_uneven(sweeps, seconds, seed, n_items):
    """Bond updates/s of the CPU oracle on the first items of the uneven
    workload (fresh child process, all host cores available to BLAS)."""
    cores = len(os.sched_getaffinity(0))
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I
items = I.uneven_batch({seed}, {n_items})
run = lambda it: O.bond_update(it[2], it[3], it[4], O.Config(D=it[0], r=it[1], sweeps={sweeps}))
run(items[0])
t0 = time.perf_counter(); n = 0
while n < len(items) and (n < 2 or time.perf_counter() - t0 < {seconds}):
    run(items[n]); n += 1
print(json.dumps({{"n": n, "seconds": time.perf_counter() - t0}}))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    return res["n"] / res["seconds"], res["n"], res["seconds"], cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    D, r, sweeps = args.D, args.r, args.sweeps
    times, items = [], 0
    cores = len(os.sched_getaffinity(0))
    uneven = args.workload == "uneven"
    # one step = a bounded sample of the workload on the host cores
    for i in range(args.warmup + args.steps):
        if uneven:
            rate, n, sec, cores = _oracle_rate_uneven(args.sweeps, args.ref_seconds, 5 + i, 8)
        else:
            rate, n, sec, cores, _ = _oracle_rate(D, r, sweeps, args.ref_seconds, 5 + i,
                                                  max_items=args.ref_items)
        if i >= args.warmup:
            times.append(sec)
            items += n
    value = items / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "bond updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {**(uneven_config(args, "fp64 oracle (CPU)") if uneven
                       else workload_config(args, "fp64 oracle (CPU)")),
                   "reference_sample": f"each step times the oracle on a bounded sample of the "
                                       f"workload: {items // max(1, args.steps)} items on "
                                       f"average (at most {args.ref_items} per step, "
                                       f"{args.ref_seconds:g} s), not the whole batch"},
        "cpu_baseline": {"value": value, "unit": "bond updates/s", "cores": cores,
                         "kind": "oracle",
                         "sample": (f"{items} bond updates of the uneven workload" if uneven else
                                    f"{items} D={D} bond updates") + f" over {args.steps} steps"},
        "e2e": {"value": value, "unit": "bond updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def workload_config(args, precision):
    return {"workload": f"batched NTU bond updates, D={args.D} d=2 r={args.r}, "
                        f"exp(-i 0.01 ZZ), {args.sweeps} ALS sweeps",
            "D": args.D, "d": 2, "r": args.r, "batch_per_gpu": args.batch,
            "sweeps": args.sweeps, "precision": precision, "seed": 5,
            "l2": "flushed (256 MB write) before every timed step"}


def uneven_config(args, precision):
    return {"workload": f"uneven batch: {args.batch} independent NTU bond updates, D uniform in "
                        f"3..8, r in {{2, 4}} (exp(-i 0.01 ZZ) / exp(-i 0.01 (XX+YY+ZZ))), "
                        f"complex64 draws, {args.sweeps} ALS sweeps",
            "batch_per_gpu": args.batch, "sweeps": args.sweeps, "precision": precision,
            "seed": 5, "l2": "flushed (256 MB write) before every timed step"}


def run_uneven(args):
    """The uneven workload: items grouped by kind (D, r), the kinds' batched
    updates forked onto one stream per kind and replayed as one CUDA graph;
    compared with the same grouped enqueue without the graph and with one
    launch sequence per bond."""
    import torch
    from paper_2107_06635_gb300 import ntu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, dist, "cuda")

    B, S = args.batch, args.sweeps
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    items = I.uneven_batch(rank_seed(rank), B)
    kinds = sorted({(it[0], it[1]) for it in items})
    caps = [sum(1 for it in items if (it[0], it[1]) == k) for k in kinds]
    prec = {"bf16x3": ntu.NTU_MIXED_BF16X3, "fp32": ntu.NTU_MIXED_FP32,
            "fp64": ntu.NTU_FP64}[args.precision]

    def timed(ub, mode, steps, warmup):
        ts, launches = [], 0
        for i in range(warmup + steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ub.run(mode)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            if i >= warmup:
                ts.append(e0.elapsed_time(e1))
                launches += ub.last_launch_count()
        ub.sync()
        return max_over_ranks(statistics.mean(ts)), launches

    def make(p):
        ub = ntu.UnevenBatch(kinds, caps, sweeps=S, precision=p,
                             tau_kmax=15 if p == ntu.NTU_FP64 else 8, stream=stream.cuda_stream)
        ub.stage(items)
        return ub

    ub = make(prec)
    tuning = None
    if not args.no_tune:
        # the schedule of the critical path: the kind with the most work per
        # item (the ALS grows as (D r)^4 D); searched in graph replay, as timed
        from paper_2107_06635_gb300 import autotune
        heavy = max(range(len(kinds)), key=lambda k: (kinds[k][0] * kinds[k][1]) ** 4 * kinds[k][0])
        tuning = autotune.tune_uneven(ub, kinds, heavy, stream, reps=3)
    clocks = ClockSampler(local)
    clocks.start()
    ms_graph, launches = timed(ub, ub.GRAPH, args.steps, args.warmup)
    clk = clocks.stop()
    ms_grouped, _ = timed(ub, ub.GROUPED, args.steps, 1)
    ms_item, _ = timed(ub, ub.PER_ITEM, max(1, min(args.steps, 2)), 1)
    _, _, info = ub.fetch(items)

    # end to end through the host call (graph replay, copies in and out)
    t_e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ub.update(items, use_graph=True)
        dt = time.perf_counter() - t0
        barrier()
        if i >= args.warmup:
            t_e2e.append(dt)
    e2e_s = max_over_ranks(statistics.mean(t_e2e))
    ub.close()

    fp64 = None
    if not args.no_fp64 and prec != ntu.NTU_FP64:
        u64 = make(ntu.NTU_FP64)
        ms64, _ = timed(u64, u64.GRAPH, args.fp64_steps, 1)
        u64.close()
        fp64 = {"value": job_rate(world, B, ms64), "unit": "bond updates/s", "ms_per_step": ms64}
    if rank != 0:
        return
    value = job_rate(world, B, ms_graph)
    env_total = sum(env_flops(it[0], it[1]) for it in items)
    peaks = measured_peaks()
    roof = env_roof(args.precision, env_total / (ms_graph / 1e3), peaks)
    roof["kernel"] = ("whole step: environment flops of every item over the step time "
                      "(a lower bound on the tensor-core kernels' own rate)")
    roof["traffic"] = None
    cpu = None
    if not args.no_cpu_baseline:
        rate, n, sec, cores = _oracle_rate_uneven(S, args.cpu_seconds, 5, 64)
        cpu = {"value": rate, "unit": "bond updates/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {n} bond updates of the uneven workload in {sec:.1f} s "
                         f"(numpy/BLAS, {cores} threads)"}
    in_b = sum(it[2].size + it[3].size + it[4].size for it in items) * 16
    out_b = sum(it[2].size + it[3].size for it in items) * 16 + B * 4 * 8
    line = {
        "metric": METRIC, "value": value, "unit": "bond updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": DTYPE_BF16X3, "fp32": DTYPE_FP32, "fp64": "c128"}[args.precision],
        "data": "synthetic",
        "config": uneven_config(args, args.precision),
        "kinds": {f"D{k[0]}r{k[1]}": c for k, c in zip(kinds, caps)},
        "tuning": tuning,
        "roofline": roof,
        "grouped_no_graph": {"value": job_rate(world, B, ms_grouped), "ms_per_step": ms_grouped},
        "per_bond_launches": {"value": job_rate(world, B, ms_item), "ms_per_step": ms_item},
        "speedup_vs_per_bond": ms_item / ms_graph,
        "fp64_path": fp64,
        "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
        "delta_median": float(np.median(info[:, 1])),
        "e2e": {"value": job_rate(world, B, 1e3 * e2e_s), "unit": "bond updates/s",
                "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch
    from paper_2107_06635_gb300 import ntu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, dist, "cuda")

    D, r, B, S = args.D, args.r, args.batch, args.sweeps
    # one non-default stream shared by torch (events, L2 flush) and the library
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    Ta_h, Tb_h, G_h = I.batch_items(rank_seed(rank), B, 2, D, I.zz_gate(0.01))
    Ta = torch.from_numpy(Ta_h).cuda()
    Tb = torch.from_numpy(Tb_h).cuda()
    G = torch.from_numpy(G_h).cuda()
    Ta_o, Tb_o = torch.empty_like(Ta), torch.empty_like(Tb)
    info = torch.empty((B, 4), dtype=torch.float64, device="cuda")

    def measure(precision, steps, warmup, kmax, tune=False):
        ctx = ntu.Context(D, 2, 1, r, S, precision, 4, kmax, B, stream=stream.cuda_stream)
        ctx.tuning = None
        if args.tuning:
            ctx.set_tuning(**json.loads(args.tuning))
            ctx.tuning = {"chosen": json.loads(args.tuning), "source": "--tuning"}
        elif tune:
            ctx.tuning = tuned(ctx, precision)
        ctx.set_profiling(True)
        t_step, stages, launches = [], [], 0
        for i in range(warmup + steps):
            if i == warmup:
                ctx.solver_paths()            # count the timed steps only
            flush.fill_(float(i))
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.batch_update_dev(B, Ta, Tb, G, Ta_o, Tb_o, info)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            if i >= warmup:
                t_step.append(e0.elapsed_time(e1))
                stages.append(ctx.stage_times())
                launches += ctx.last_launch_count()
        ctx.sync()
        ctx.paths = ctx.solver_paths()
        return ctx, t_step, np.mean(stages, axis=0), launches

    def tuned(ctx, precision):
        """The workload's schedule from the autotuner: the cached choice for
        this device and workload, else a search (timed before the measured
        region), whose result is cached."""
        from paper_2107_06635_gb300 import autotune
        dev = torch.cuda.get_device_name()
        key = {"D": D, "r": r, "d": 2, "batch": B, "sweeps": S, "precision": int(precision),
           "library": 3}
        rec = None if args.retune else autotune.lookup(dev, key)
        if rec is not None:
            ctx.set_tuning(**rec["chosen"])
            return {**rec, "source": "cache"}
        rec = autotune.tune_batch(ctx, B, Ta, Tb, G, Ta_o, Tb_o, info, stream, reps=3)
        autotune.remember(dev, key, rec)
        return {**rec, "source": "search"}

    head = {"bf16x3": ntu.NTU_MIXED_BF16X3, "fp32": ntu.NTU_MIXED_FP32,
            "fp64": ntu.NTU_FP64}[args.precision]
    clocks = ClockSampler(local)
    clocks.start()
    ctx, t_mixed, st_mixed, launches = measure(head, args.steps, args.warmup,
                                               15 if head == ntu.NTU_FP64 else 8,
                                               tune=not args.no_tune)
    tuning = ctx.tuning
    clk = clocks.stop()
    ms_mixed = max_over_ranks(statistics.mean(t_mixed))
    value = job_rate(world, B, ms_mixed)
    delta_mixed = info[:, 1].cpu().numpy()
    paths_mixed = ctx.paths

    # end to end through the host-pointer call: pinned inputs in, results out
    pin = lambda a: torch.from_numpy(a).pin_memory()
    hTa, hTb, hG = pin(Ta_h), pin(Tb_h), pin(G_h)
    hA = torch.empty_like(hTa).pin_memory()
    hB = torch.empty_like(hTb).pin_memory()
    hI = torch.empty((B, 4), dtype=torch.float64).pin_memory()
    t_e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ctx._ck(ctx.lib.ntu_batch_update_host(ctx.h, B, hTa.data_ptr(), hTb.data_ptr(),
                                              hG.data_ptr(), hA.data_ptr(), hB.data_ptr(),
                                              hI.data_ptr()))
        dt = time.perf_counter() - t0
        barrier()
        if i >= args.warmup:
            t_e2e.append(dt)
    e2e_s = max_over_ranks(statistics.mean(t_e2e))
    h2d = (Ta_h.nbytes + Tb_h.nbytes + G_h.nbytes)
    d2h = (Ta_h.nbytes + Tb_h.nbytes + B * 4 * 8)
    sample_idx = sorted({0, B // 2, B - 1})
    gpu_sample = gpu_sample_items(ctx, torch, ntu, Ta, Tb, G, Ta_o, Tb_o, info, sample_idx)
    ctx.close()
    del ctx

    # the other precisions on the same GPU, same batch
    # FP64 / FP32 ceilings of the SIMT environment paths, measured here
    gemm_peaks = measure_gemm_peaks()
    others = {}
    names = {ntu.NTU_MIXED_BF16X3: "bf16x3_path", ntu.NTU_MIXED_FP32: "fp32_env_path",
             ntu.NTU_FP64: "fp64_path"}
    for prec in (ntu.NTU_MIXED_BF16X3, ntu.NTU_MIXED_FP32, ntu.NTU_FP64):
        if prec == head or (prec == ntu.NTU_FP64 and args.no_fp64):
            continue
        cx, tt, st, _ = measure(prec, args.fp64_steps, 1, 15 if prec == ntu.NTU_FP64 else 8)
        ms = max_over_ranks(statistics.mean(tt))
        env_rate = B * env_flops(D, r) / (st[1] / 1e3)
        others[names[prec]] = {
            "value": job_rate(world, B, ms), "unit": "bond updates/s", "ms_per_step": ms,
            "env_tflops": env_rate / 1e12,
            "env_roofline": env_roof("fp64" if prec == ntu.NTU_FP64 else "fp32", env_rate,
                                     gemm_peaks),
            "stage_ms": dict(zip(["gate_qr", "env", "repair", "als", "recompose"],
                                 [round(float(x), 3) for x in st]))}
        cx.close()
    fp64 = others.get("fp64_path")

    # the metric names D=6 as well: the same batch and sweeps at D=6, this
    # precision and the FP64 path (device-resident, L2 flushed per step)
    def measure_d(Dm, prec, steps, warmup):
        ta_h, tb_h, g_h = I.batch_items(rank_seed(rank), B, 2, Dm, I.zz_gate(0.01))
        ta, tb, gg = (torch.from_numpy(x).cuda() for x in (ta_h, tb_h, g_h))
        oa, ob = torch.empty_like(ta), torch.empty_like(tb)
        inf = torch.empty((B, 4), dtype=torch.float64, device="cuda")
        cx = ntu.Context(Dm, 2, 1, r, S, prec, 4, 15 if prec == ntu.NTU_FP64 else 8, B,
                         stream=stream.cuda_stream)
        ts = []
        for i in range(warmup + steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cx.batch_update_dev(B, ta, tb, gg, oa, ob, inf)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            if i >= warmup:
                ts.append(e0.elapsed_time(e1))
        cx.sync()
        cx.close()
        ms = max_over_ranks(statistics.mean(ts))
        return {"value": job_rate(world, B, ms), "unit": "bond updates/s", "ms_per_step": ms}

    def measure_cell(Dc, prec, steps=20, warmup=3):
        """The unit-cell Trotter step of one NTU Trotter step of the two-site
        cell (ntu_step: four bond updates, gate exp(-i 0.01 ZZ), 10 sweeps,
        iid complex site tensors from seed 1; host gates in, deltas out,
        synchronised) with its launches replayed from one CUDA graph and
        issued one by one; wall time per step on the host."""
        gates2 = [I.zz_gate(0.01)] * 4
        gate1 = None
        out = {"D": Dc, "precision": int(prec),
               "workload": f"one NTU Trotter step of the 2-site cell, D={Dc}, seed 1, "
                           "exp(-i 0.01 ZZ), 10 sweeps"}
        for graphs in (True, False):
            cx = ntu.Context(Dc, 2, 1, r, S, prec, 4, 15 if prec == ntu.NTU_FP64 else 8, 1,
                             stream=stream.cuda_stream)
            cx.set_graphs(graphs)
            cx.set_state(*I.random_pair(1, 2, Dc))
            for _ in range(warmup):
                cx.step(gates2, gate1)
            t0 = time.perf_counter()
            for _ in range(steps):
                cx.step(gates2, gate1)
            dt = (time.perf_counter() - t0) / steps
            out["graph" if graphs else "direct"] = {
                "ms_per_step": 1e3 * dt, "bond_updates_per_s": 4 / dt,
                "launches_per_step": cx.last_launch_count()}
            cx.close()
        out["speedup_graph"] = out["direct"]["ms_per_step"] / out["graph"]["ms_per_step"]
        return out

    cell = None if args.no_cell else measure_cell(3, ntu.NTU_FP64)

    d6 = None
    if D != 6 and not args.no_d6:
        d6 = {"D": 6, "batch_per_gpu": B, "path": args.precision,
              **measure_d(6, head, args.steps, args.warmup)}
        if not args.no_fp64 and head != ntu.NTU_FP64:
            f6 = measure_d(6, ntu.NTU_FP64, args.fp64_steps, 1)
            d6["fp64_path"] = f6
            d6["speedup_vs_fp64"] = d6["value"] / f6["value"]

    if rank != 0:
        return

    als_ms = float(st_mixed[3])
    achieved = B * als_flops(D, r, S) / (als_ms / 1e3)
    als_pk, als_pk_src = als_peak(args.precision, gemm_peaks)
    env_achieved = B * env_flops(D, r) / (float(st_mixed[1]) / 1e3)
    cpu, cpu_all, accuracy = None, None, None
    if not args.no_cpu_baseline:
        # the oracle single-threaded (one bond update per core, the plan for
        # this workload); its first items are the accuracy sample
        kmax = 15 if args.precision == "fp64" else 8
        rate, n, sec, th, kept = _oracle_rate(D, r, S, args.cpu_seconds, rank_seed(rank),
                                              max_items=64, threads=1, keep=sample_idx,
                                              batch=B, tau_kmax=kmax)
        cpu = {"value": rate, "unit": "bond updates/s", "cores": th, "kind": "oracle",
               "sample": f"{n} of the D={D} workload's bond updates in {sec:.1f} s "
                         f"(numpy/BLAS, 1 thread)"}
        rate, n, sec, th, _ = _oracle_rate(D, r, S, args.cpu_seconds / 2, rank_seed(rank),
                                           max_items=64, tau_kmax=kmax)
        cpu_all = {"value": rate, "unit": "bond updates/s", "cores": th, "kind": "oracle",
                   "sample": f"{n} of the D={D} workload's bond updates in {sec:.1f} s "
                             f"(numpy/BLAS, {th} threads)"}
        accuracy = accuracy_vs_oracle(gpu_sample, kept, sample_idx)
    peaks = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": "bond updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": DTYPE_BF16X3, "fp32": DTYPE_FP32, "fp64": "c128"}[args.precision],
        "data": "synthetic",
        "config": workload_config(args, {
            "bf16x3": PRECISION_BF16X3, "fp32": PRECISION_FP32,
            "fp64": "FP64 throughout"}[args.precision]),
        "roofline": {"kernel": ("ALS stage (Fig. 5): k_als with its streaming inputs k_gmax, "
                                "k_gsplit, k_oz_slice"), "bound": "alu",
                     "achieved": achieved / 1e12, "peak": als_pk / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / als_pk,
                     "traffic": als_traffic(args.precision, D, r, S, B),
                     "peak_source": als_pk_src},
        "env_roofline": env_roof(args.precision, env_achieved, {**peaks, **gemm_peaks}),
        "measured_gemm_peaks": {k: round(v, 2) for k, v in gemm_peaks.items()},
        "stage_ms": dict(zip(["gate_qr", "env", "repair", "als", "recompose"],
                             [round(float(x), 3) for x in st_mixed])),
        "delta_median": float(np.median(delta_mixed)),
        "tuning": tuning,
        "solver_paths": paths_mixed,
        **others,
        "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
        "d6": d6,
        "cell_step": cell,
        "e2e": {"value": job_rate(world, B, 1e3 * e2e_s), "unit": "bond updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "accuracy_vs_oracle": accuracy,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def gpu_sample_items(ctx, torch, ntu, Ta, Tb, G, Ta_o, Tb_o, info, idx):
    """For the sampled items of the measured batch: the repaired metric g
    from the stage calls (gate + QR, environment, repair) on the same
    context, the batch's A', B' and [eps, delta, eps0, tau], and the cluster
    estimator <sigma_x> on site A of the updated pair (all on the GPU)."""
    n = len(idx)
    sel = torch.tensor(idx, device="cuda")
    ta, tb, gg = Ta[sel].contiguous(), Tb[sel].contiguous(), G[sel].contiguous()
    m, K = ctx.d_p * ctx.D ** 3, ctx.K
    c128 = dict(dtype=torch.complex128, device="cuda")
    QA, QB = torch.empty((n, m, K), **c128), torch.empty((n, m, K), **c128)
    RA, RB = torch.empty((n, K, K), **c128), torch.empty((n, K, K), **c128)
    g = torch.empty((n, K * K, K * K), **c128)
    diag = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.batch_gate_qr_dev(n, ta, tb, gg, QA, RA, QB, RB)
    ctx.batch_env_dev(n, ta, tb, QA, QB, g)
    ctx.batch_repair_dev(n, g, diag)
    ctx.sync()
    A, Bs = Ta_o[sel].cpu().numpy(), Tb_o[sel].cpu().numpy()
    sx = []
    for j in range(n):
        ctx.set_state(A[j], Bs[j])
        sx.append(ctx.measure(0, I.pauli("X")).real)
    return {"g": g.cpu().numpy(), "A": A, "B": Bs, "info": info[sel].cpu().numpy(),
            "sx": np.array(sx)}


def accuracy_vs_oracle(gpu, kept, idx):
    """Errors of the GPU path against the FP64 oracle on the sampled items:
    relative Frobenius error of the repaired metric g, relative error of the
    NTU error delta, relative error of the updated two-site state A'B'
    (contracted over the bond) and |delta <sigma_x>| of the cluster estimator
    on the updated pair."""
    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    pair = lambda a, b: np.einsum("plurn,qrvwx->plunqvwx", a, b)
    g_err, d_err, p_err, x_err = [], [], [], []
    for j, i in enumerate(idx):
        g_err.append(rel(gpu["g"][j], kept[f"g{i}"]))
        d_ref = kept[f"d{i}"][0]
        d_err.append(abs(gpu["info"][j, 1] - d_ref) / d_ref)
        p_err.append(rel(pair(gpu["A"][j], gpu["B"][j]), pair(kept[f"A{i}"], kept[f"B{i}"])))
        x_err.append(abs(gpu["sx"][j] - kept[f"x{i}"][0]))
    return {"items": idx, "g_rel_frob_max": max(g_err), "delta_rel_max": max(d_err),
            "pair_rel_max": max(p_err), "sx_abs_max": max(x_err),
            "tolerances": {"g_rel_frob": "1e-4 mixed / 1e-10 fp64", "delta_rel": 1e-2,
                           "pair_rel": 1e-4}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--D", type=int, default=8)
    ap.add_argument("--r", type=int, default=2)
    ap.add_argument("--batch", type=int, default=None, help="default 912 (uniform), 512 (uneven)")
    ap.add_argument("--sweeps", type=int, default=None, help="default 10 (uniform), 8 (uneven)")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-d6", action="store_true", help="skip the D=6 lines of the metric")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    ap.add_argument("--ref-items", type=int, default=8,
                    help="most items the reference arm times per step")
    ap.add_argument("--no-cell", action="store_true", help="skip the unit-cell step line")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the automatic schedule instead of the autotuner's choice")
    ap.add_argument("--retune", action="store_true", help="search again, ignoring the cache")
    ap.add_argument("--tuning", default=None,
                    help='a fixed ntu_set_tuning choice as JSON, e.g. \'{"als_split": 1}\' '
                         '(replaces the autotuner)')
    ap.add_argument("--workload", default="uniform", choices=["uniform", "uneven"],
                    help="uniform: the D=8 batch (default); uneven: D in 3..8, r in {2, 4}")
    args = ap.parse_args()
    uneven = args.workload == "uneven"
    if args.batch is None:
        args.batch = 512 if uneven else 912
    if args.sweeps is None:
        args.sweeps = 8 if uneven else 10
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
