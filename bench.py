#!/usr/bin/env python
"""Benchmark of the two-level sampling-based clustering on GB300.

One step = one whole job on one batch of synthetic input: min-max scaling, the landmark
peel into subclusters, Lloyd on every subcluster, Lloyd on the pooled local centers and
the SSE of every point (all kernels of the library, recorded once into a CUDA graph and
replayed).  Workload: 2^20 points, d=16, 64 Gaussian blobs (sigma ~ U[0.2, 1]) + 1%
uniform outliers, subclusters of 4096 (256 of them), 64 local centers, 25 Lloyd
iterations, final k=64.

Arithmetic: by default the assignment runs on the tensor cores (--prec tc: TF32x3 or
BF16x3 contraction, near ties re-decided in float32), which assigns exactly as the float32
direct form does; --prec fp32 runs the float32 direct kernel.

Metric: Lloyd distance evaluations per second of the whole job,
    sum over subclusters of |s| * k_eff * iters + pooled * final_k * iters,
divided by the job's device time (so peel, scaling and SSE count against it).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank runs its own independent job (another seed): weak scaling,
no collective on the data path; rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1412_1947_gb300 import synth  # noqa: E402

METRIC = "Lloyd dist-evals/s"
UNIT = "dist-evals/s"
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense TF32 : BF16 tensor rate of the part


def tc_mode(prec: str, w: synth.Workload) -> str:
    """The arithmetic the local Lloyd runs in: "tc" is the split mode the library picks for
    the shape (TF32x3 where its tiles fit one CTA's shared memory, else BF16x3)."""
    if prec != "tc":
        return prec
    return "tf32x3" if w.d <= 32 or (w.d == 64 and w.local_k <= 16) else "bf16x3"


def measured_peaks():
    """The machine's measured peaks (HBM copy GB/s; cuBLAS bf16 TFLOP/s burst and sustained),
    else the earlier GB300 measurement used as fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m["bf16_tflops"]),
                "bf16_tflops_sustained": float(m.get("bf16_tflops_sustained", m["bf16_tflops"])),
                "kind": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "kind": "fallback"}


def replica_max(x: float, dist=None) -> float:
    """The maximum of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_evals(w: synth.Workload) -> int:
    """Distance evaluations of one job (local Lloyd + final Lloyd)."""
    full, rem = divmod(w.n, w.N)
    ev = full * w.N * min(w.local_k, w.N)
    P = full * min(w.local_k, w.N)
    if rem:
        ev += rem * min(w.local_k, rem)
        P += min(w.local_k, rem)
    return (ev + P * w.final_k) * w.iters


def config_of(w: synth.Workload, extra=None):
    c = {"workload": w.name, "n": w.n, "d": w.d, "blobs": w.blobs, "N": w.N, "local_k": w.local_k,
         "final_k": w.final_k, "iters": w.iters, "outliers": w.outlier_frac,
         "l2": "flushed (256 MiB write) between timed steps", "storage": "f32"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_sample(w: synth.Workload, n_sample: int):
    # enough subclusters that the pooled local centers can seed final_k of them
    n_sample = max(n_sample, -(-w.final_k // w.local_k) * w.N)
    return synth.Workload(w.name + f"_sample{n_sample}", n=n_sample, d=w.d, blobs=w.blobs, N=w.N,
                          local_k=w.local_k, final_k=w.final_k, iters=w.iters, sigma=w.sigma,
                          outlier_frac=w.outlier_frac, seed=w.seed)


def run_oracle_once(ws: synth.Workload, raw, threads: int) -> float:
    import oracle
    t0 = time.perf_counter()
    oracle.two_level(raw, ws.N, ws.local_k, ws.final_k, ws.iters, seed=1, threads=threads)
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it, else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline(w: synth.Workload, n_sample: int):
    """The oracle on the workload's full data once (all host threads), and on an n_sample
    sample of the same recipe with one thread."""
    threads = os.cpu_count() or 1
    secs = run_oracle_once(w, w.points(), threads)
    ws = oracle_sample(w, n_sample)
    secs1 = run_oracle_once(ws, ws.points(), 1)
    return {"value": workload_evals(w) / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the whole two-level job (scale, peel, Lloyd, final Lloyd, SSE) on the full workload "
                      f"(n={w.n}, {-(-w.n // w.N)} subclusters of {w.N}), once, {secs:.2f} s, float64 C "
                      f"oracle, OpenMP over subclusters",
            "cpu": cpu_model(),
            "single_thread": {"value": workload_evals(ws) / secs1, "unit": UNIT, "seconds": secs1,
                              "sample": f"n={ws.n} points of the same recipe"}}


# ------------------------------------------------------------------ reference arm
def reference_arm(args, w: synth.Workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = args.oracle_n
    ws = oracle_sample(w, n_sample)
    raw = ws.points()
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        run_oracle_once(ws, raw, threads)
    times = [run_oracle_once(ws, raw, threads) for _ in range(args.steps)]
    ev = workload_evals(ws)
    value = ev / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, {"sample_n": ws.n}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"n={ws.n} points of the same recipe per step", "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def main_arm(args, w: synth.Workload):
    import numpy as np
    import torch

    from paper_1412_1947_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    # a stream of our own (the legacy default stream has handle 0, which the library
    # would read as "make your own stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    wr = synth.Workload(w.name, n=w.n, d=w.d, blobs=w.blobs, N=w.N, local_k=w.local_k, final_k=w.final_k,
                        iters=w.iters, sigma=w.sigma, outlier_frac=w.outlier_frac, seed=w.seed + 1000 * rank)
    raw = wr.points()
    evals = workload_evals(wr)
    seed = 12345
    prec = B.PRECISIONS[args.prec]
    x_dev = torch.from_numpy(raw).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    fma_tflops = B.pscl_measure_fp32_fma(local)
    barrier_us = B.pscl_measure_grid_barrier(local)
    ctx = B.pscl_ctx_create(local, 0, stream.cuda_stream)
    job = B.Job(x_dev, ctx=ctx)
    job.option(B.PSCL_OPT_GRAPH)
    job.option(B.PSCL_OPT_ROWS_PER_THREAD, args.rows_per_thread)
    run = lambda: job.run(wr.N, wr.local_k, wr.final_k, wr.iters, seed, prec)  # noqa: E731

    for _ in range(args.warmup):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    launches_per_step = sum(v[0] for v in job.kernel_times().values())

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()                                  # outside the timed interval
        starts[i].record(stream)
        run()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    mean_ms = replica_max(statistics.mean(step_ms), dist)
    _, _, sse = job.result(labels=False)

    # ---- end to end through the public API with host buffers: H2D of the points from
    # pinned memory, the job, D2H of the final centers and SSE, every step
    host = torch.from_numpy(raw).pin_memory()
    ctx_e = B.pscl_ctx_create(local, 0, stream.cuda_stream)
    job_e = B.Job(host, ctx=ctx_e)
    job_e.option(B.PSCL_OPT_GRAPH)
    job_e.option(B.PSCL_OPT_ROWS_PER_THREAD, args.rows_per_thread)
    for _ in range(max(1, args.warmup)):
        job_e.load(host)
        job_e.run(wr.N, wr.local_k, wr.final_k, wr.iters, seed, prec)
        job_e.result(labels=False)
    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        job_e.load(host)
        job_e.run(wr.N, wr.local_k, wr.final_k, wr.iters, seed, prec)
        c, _, sse_e = job_e.result(labels=False)
        e2e_s.append(time.perf_counter() - t0)
    e2e_mean = replica_max(statistics.mean(e2e_s), dist)
    job_e.close()
    B.pscl_ctx_destroy(ctx_e)

    # ---- per-kernel device times (events around every launch, unrecorded runs)
    job_k = B.Job(x_dev, ctx=ctx)
    job_k.option(B.PSCL_OPT_KERNEL_TIMING)
    job_k.option(B.PSCL_OPT_ROWS_PER_THREAD, args.rows_per_thread)
    kt = None
    for _ in range(2):
        flush.zero_()
        job_k.steps(wr.N, wr.local_k, wr.final_k, wr.iters, seed, prec)
        kt = job_k.kernel_times()
    rechecked, assigned = job_k.recheck_stats()
    peel_epochs, peel_passes, peel_updates, peel_barriers = job_k.peel_stats()
    phases = job_k.phase_ms()
    job_k.close()

    # ---- the plain per-subcluster float32 form on the same data
    plain = None
    if not args.no_plain:
        job_p = B.Job(x_dev, ctx=ctx)
        job_p.option(B.PSCL_OPT_PLAIN_LLOYD)
        pl_ms = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            job_p.steps(wr.N, wr.local_k, wr.final_k, wr.iters, seed)
            ph = job_p.phase_ms()
            pl_ms.append(ph)
        _, _, sse_p = job_p.result(labels=False)
        ph = pl_ms[-1]
        local_evals = evals - 0
        plain = {"form": "plain float32, one launch pair per subcluster per iteration",
                 "ms_per_job": float(sum(ph)), "local_lloyd_ms": float(ph[2]),
                 "value": evals / (float(sum(ph)) * 1e-3), "sse": sse_p, "sse_equal": sse_p == sse}
        job_p.close()
        del local_evals

    # ---- count-weighted pooling on the same data: its final SSE against the unweighted one
    job_w = B.Job(x_dev, ctx=ctx)
    job_w.option(B.PSCL_OPT_POOL_WEIGHTED)
    job_w.steps(wr.N, wr.local_k, wr.final_k, wr.iters, seed, B.PRECISIONS[args.prec])
    _, _, sse_w = job_w.result(labels=False)
    ph_w = job_w.phase_ms()
    pool_weighted = {"sse": sse_w, "sse_unweighted": sse, "sse_ratio": sse_w / sse,
                     "ms_per_job": float(sum(ph_w)), "final_lloyd_ms": float(ph_w[3])}
    job_w.close()

    job.close()
    B.pscl_ctx_destroy(ctx)

    # ---- rooflines: the dominant kernel, and the assignment against its own measured peak
    pk = measured_peaks()
    of = "of measured" if pk["kind"] == "measured" else "of fallback"
    S = -(-wr.n // wr.N)

    def hbm_roof(kname, byts):
        n_l, t_ms = kt[kname]
        r = {"kernel": kname, "bound": "hbm", "achieved": byts / (t_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
             "unit": "GB/s", "peak_kind": f"{of} HBM copy", "per_launch_ms": t_ms / n_l, "launches": n_l,
             "traffic": None, "algorithmic_bytes": byts}
        r["frac"] = r["achieved"] / r["peak"]
        return r

    def assign_roof():
        n_l, t_ms = kt["lloyd_assign"]
        flops = 2 * wr.d * evals                      # the contraction: 2d flops per evaluation
        tc = args.prec != "fp32" and assigned > 0
        mode = tc_mode(args.prec, wr)
        if tc:
            peak = pk["bf16_tflops"] * (1.0 if mode.startswith("bf16") else TF32_PER_BF16)
            kind = f"{of} cuBLAS bf16 burst" + ("" if mode.startswith("bf16") else " x nominal tf32/bf16")
        else:
            peak = fma_tflops
            kind = "measured float32 FMA rate (pscl_measure_fp32_fma, 2 flop per FMA)"
        r = {"kernel": f"k_tc_assign (tcgen05, {mode})" if tc else "k_lloyd_assign (float32 direct)",
             "bound": "tensor" if tc else "alu", "achieved": flops / (t_ms * 1e-3) / 1e12, "peak": peak,
             "unit": "TFLOP/s", "peak_kind": kind, "per_launch_ms": t_ms / n_l, "launches": n_l, "traffic": None,
             "algorithmic_flops": flops,
             # d*4/k bytes per evaluation: each point read once per iteration serves k distances
             "achieved_gbs": evals * wr.d * 4 / wr.local_k / (t_ms * 1e-3) / 1e9}
        if tc and "lloyd_sums" in kt:
            r["sums_pass_ms"] = kt["lloyd_sums"][1]
        r["frac"] = r["achieved"] / r["peak"]
        return r

    name = max(kt.items(), key=lambda kv: kv[1][1])[0]
    if name == "peel":
        # one read of the remaining points per round: sum over rounds of n_r * d * 4 bytes
        roof = hbm_roof("peel", sum(wr.n - r * wr.N for r in range(S)) * wr.d * 4)
        roof["us_per_round"] = 1e3 * kt["peel"][1] / S
    elif name == "lloyd_assign":
        roof = assign_roof()
    else:
        roof = hbm_roof(name, wr.n * wr.d * 4 * 2)

    value = evals * world / (mean_ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else tc_mode(args.prec, wr) + "+f32",
            "data": "synthetic",
            "near_ties": {"rechecked_rows": rechecked, "tensor_core_rows": assigned},
            "peel": {"epochs": peel_epochs, "distance_passes": peel_passes, "key_updates": peel_updates},
            "config": config_of(wr, {"parallelism": f"replicas{world}" if world > 1 else "single"}),
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
            "sse": sse,
            "e2e": {"value": evals * world / e2e_mean, "unit": UNIT,
                    "h2d_bytes_per_step": int(raw.nbytes), "d2h_bytes_per_step": wr.final_k * wr.d * 4 + 8},
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roof,
            "roofline_assign": assign_roof(),
            # the peel's latency floor: its grid barriers at the measured cost of one
            "peel_latency": {"bound": "grid barriers", "grid_barrier_us": barrier_us, "barriers": peel_barriers,
                             "floor_ms": peel_barriers * barrier_us / 1e3, "peel_ms": kt["peel"][1],
                             "frac": peel_barriers * barrier_us / 1e3 / kt["peel"][1],
                             "peak_kind": "measured (pscl_measure_grid_barrier, the peel's barrier in its launch shape)"},
            "kernels_ms": {k: round(v[1], 4) for k, v in kt.items()},
            "kernel_launches": {k: v[0] for k, v in kt.items()},
            "phase_ms": {"scale": float(phases[0]), "peel": float(phases[1]), "local_lloyd": float(phases[2]),
                         "final_lloyd": float(phases[3]), "sse": float(phases[4])},
            "lloyd_only_value": evals / (float(phases[2] + phases[3]) * 1e-3),
            "plain_fp32": plain, "pool_weighted": pool_weighted, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, args.oracle_n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main_uneven(args):
    """The uneven batch: 2048 independent instances, sizes log-uniform in [256, 65536],
    d = 32, k = max(8, size / 256), 25 Lloyd iterations, every instance min-max scaled on
    its own; one graph-recorded run of all instances per step, work-unit shape from the
    autotuner.  Printed as its own line (not the default workload)."""
    import numpy as np
    import torch

    import oracle
    from paper_1412_1947_gb300 import binding as B

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    iters, seed = 25, 777
    prec = B.PRECISIONS[args.prec]
    parts, ks = synth.uneven_batch()
    sizes = np.array([len(p) for p in parts], np.int64)
    keff = np.minimum(np.array(ks, np.int64), sizes)
    raw = np.ascontiguousarray(np.concatenate(parts), np.float32)
    evals = int((sizes * keff).sum()) * iters
    x_dev = torch.from_numpy(raw).to(dev)
    ctx = B.pscl_ctx_create(0, 0, stream.cuda_stream)
    b = B.Batch(x_dev, sizes, ks, ctx=ctx)
    unit_rows, rpt, _ = b.tune(2, prec)
    for _ in range(args.warmup):
        b.run(iters, seed, prec)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(0)
    clk.start()
    for i in range(args.steps):
        starts[i].record(stream)
        b.run(iters, seed, prec)
        ends[i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    step_ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
    mean_ms = statistics.mean(step_ms)
    launches_per_step = b.launches()
    _, _, sse = b.result(labels=False)
    # the Lloyd iterations alone (unrecorded run, events around them)
    b.option(B.PSCL_OPT_GRAPH, 0)
    b.run(iters, seed, prec)
    lloyd_ms = b.lloyd_ms()
    # the plain form: one launch pair per instance and iteration
    plain = None
    if not args.no_plain:
        b.option(B.PSCL_OPT_PLAIN_LLOYD, 1)
        b.run(iters, seed, B.PSCL_PREC_FP32)
        pl_ms = b.lloyd_ms()
        _, _, sse_p = b.result(labels=False)
        plain = {"form": "plain float32, one launch pair per instance per iteration", "lloyd_ms": pl_ms,
                 "value": evals / (pl_ms * 1e-3), "sse_equal": bool(np.array_equal(sse_p, sse))}
        b.option(B.PSCL_OPT_PLAIN_LLOYD, 0)
    b.option(B.PSCL_OPT_GRAPH, 1)
    # end to end: pinned host points in, per-instance SSE out, every step
    host = torch.from_numpy(raw).pin_memory()
    e2e_s = []
    for i in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.load(host)
        b.run(iters, seed, prec)
        _, _, _ = b.result(labels=False)
        if i:
            e2e_s.append(time.perf_counter() - t0)
    e2e_mean = statistics.mean(e2e_s)
    d = raw.shape[1]
    flops = evals * 2 * d                 # the contraction: 2d flops per distance evaluation
    if args.prec == "fp32":
        roof = {"kernel": "Lloyd iterations (k_lloyd_assign + finalize)", "bound": "alu",
                "achieved": flops / (lloyd_ms * 1e-3) / 1e12, "peak": B.pscl_measure_fp32_fma(0),
                "unit": "TFLOP/s", "peak_kind": "measured float32 FMA rate (pscl_measure_fp32_fma, 2 flop per FMA)",
                "traffic": None}
    else:
        mode = tc_mode(args.prec, synth.MEDIUM)       # d = 32: TF32x3 under "tc"
        pk = measured_peaks()
        roof = {"kernel": f"Lloyd iterations (k_tc_assign {mode} + k_tc_sums + finalize)", "bound": "tensor",
                "achieved": flops / (lloyd_ms * 1e-3) / 1e12,
                "peak": pk["bf16_tflops"] * (1.0 if mode.startswith("bf16") else TF32_PER_BF16), "unit": "TFLOP/s",
                "peak_kind": ("of measured" if pk["kind"] == "measured" else "of fallback") + " cuBLAS bf16 burst"
                             + ("" if mode.startswith("bf16") else " x nominal tf32/bf16"),
                "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {"metric": METRIC, "value": evals / (mean_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else tc_mode(args.prec, synth.MEDIUM) + "+f32",
            "data": "synthetic",
            "config": {"workload": "uneven2048_d32_k8to256_it25", "instances": len(sizes), "rows": int(sizes.sum()),
                       "d": d, "iters": iters, "l2": "inputs (3 GB) larger than L2",
                       "tuned": {"unit_rows": unit_rows, "rows_per_thread": "1" if rpt else "default"}},
            "lloyd_ms": lloyd_ms, "lloyd_only_value": evals / (lloyd_ms * 1e-3), "sse_sum": float(sse.sum()),
            "e2e": {"value": evals / e2e_mean, "unit": UNIT, "h2d_bytes_per_step": int(raw.nbytes),
                    "d2h_bytes_per_step": int(8 * len(sizes))},
            "gpu_launches": int(launches_per_step * args.steps), "roofline": roof, "plain_fp32": plain,
            "clocks": clocks}
    if not args.no_cpu:
        # the oracle, single-threaded, on instances in order while they fit ~1e8 distance evaluations
        budget, ev_s, t_s, used = 1e8, 0, 0.0, 0
        for i, (p, k) in enumerate(zip(parts, ks)):
            e = len(p) * min(k, len(p)) * iters
            if ev_s + e > budget:
                continue                    # instances that would overrun the sample
            xs, _, _ = oracle.scale(p)
            t0 = time.perf_counter()
            oracle.lloyd_seeded(xs, k, iters, seed, 0, i)
            t_s += time.perf_counter() - t0
            ev_s += e
            used += 1
        line["cpu_baseline"] = {"value": ev_s / t_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{used} instances taken in order while within 1e8 distance evaluations "
                                          f"({ev_s:.3g} in all), scaling + seeded Lloyd each"}
    b.close()
    B.pscl_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def main_serving(args):
    """The job server under load: a stream of two-level jobs of mixed shapes (n log-uniform
    in [1e4, --serve-n-max], d in {8, 32, 128}, final k log-uniform in [8, 1024], N = n/64, 25
    iterations), points generated on the device; one saturated pass (all jobs submitted at
    once) gives the peak jobs/s, then Poisson arrivals at 0.5x and 0.8x of it give the
    latency percentiles.  Printed as its own line (not the default workload)."""
    import random
    import threading

    import numpy as np
    import torch

    from paper_1412_1947_gb300 import binding as B

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    jobs = synth.serving_stream(args.serve_jobs, synth.BASE_SEED + 4, n_range=(1e4, args.serve_n_max))
    prec = B.PRECISIONS[args.prec]
    pts = [synth.mixture_device(j["n"], j["d"], j["blobs"], j["seed"], dev) for j in jobs]
    pts = [x.to(torch.bfloat16) if j["bf16"] else x for j, x in zip(jobs, pts)]
    torch.cuda.synchronize()
    budget = 150 << 30
    srv = B.Server(slots=args.serve_slots, hbm_budget_bytes=budget)

    def run_pass(rate):
        """Submits every job (all at once when rate is None, else Poisson arrivals at
        `rate` jobs/s); returns (wall seconds, latencies ms, results)."""
        tickets = [None] * len(jobs)
        rnd = random.Random(11)
        t0 = time.perf_counter()

        def submitter():
            for i, (j, x) in enumerate(zip(jobs, pts)):
                if rate:
                    time.sleep(rnd.expovariate(rate))
                tickets[i] = srv.submit(x, j["N"], j["local_k"], j["final_k"], j["iters"], j["seed"], prec=prec)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        lat, res = [], []
        for t in tickets:
            srv.wait(t)
            c, _, sse, times = srv.fetch(t)
            lat.append(float(times[2]))
            res.append((c, sse))
        return time.perf_counter() - t0, lat, res

    run_pass(None)                                    # warm-up (allocator pool, kernels)
    wall, lat_sat, res = run_pass(None)
    peak = len(jobs) / wall
    st = srv.stats()
    passes = {}
    for f in (0.5, 0.8):
        w, lat, _ = run_pass(f * peak)
        lat = sorted(lat)
        passes[f"{f}x"] = {"offered_jobs_per_s": f * peak, "jobs_per_s": len(jobs) / w,
                           "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}
    srv.close()
    # a sample of the jobs again, each alone: the served results must be the same
    same = 0
    sample = list(range(0, len(jobs), max(1, len(jobs) // 10)))
    for i in sample:
        j = jobs[i]
        with B.Job(pts[i]) as jb:
            jb.run(j["N"], j["local_k"], j["final_k"], j["iters"], j["seed"], prec)
            c, _, sse = jb.result(labels=False)
        same += int(np.array_equal(c, res[i][0]) and sse == res[i][1])
    ls = sorted(lat_sat)
    evals = sum((j["n"] * j["local_k"] + -(-j["n"] // j["N"]) * j["local_k"] * j["final_k"]) * j["iters"]
                for j in jobs)
    line = {"metric": "serving jobs/s", "value": peak, "unit": "jobs/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f32" if args.prec == "fp32" else args.prec + " (split mode per shape) + f32")
                     + " (bf16 storage for half the jobs)",
            "data": "synthetic (generated on the device)",
            "config": {"workload": f"serving{len(jobs)}_n1e4to{args.serve_n_max:.0e}_d8-32-128_k8to1024".replace("+0", ""),
                       "jobs": len(jobs),
                       "slots": args.serve_slots, "hbm_budget_bytes": budget, "iters": 25,
                       "bf16_jobs": sum(j["bf16"] for j in jobs),
                       "points": int(sum(j["n"] for j in jobs)),
                       "note": "n log-uniform in [1e4, %.0e]" % args.serve_n_max},
            "saturated": {"jobs_per_s": peak, "p50_ms": ls[len(ls) // 2],
                          "p99_ms": ls[min(len(ls) - 1, int(0.99 * len(ls)))],
                          "dist_evals_per_s": evals / wall, "max_running": st["max_running"],
                          "peak_bytes": st["peak_bytes"]},
            "poisson": passes, "alone_equal": f"{same}/{len(sample)}"}
    print(json.dumps(line), flush=True)


# The paper's timing tables (Table 2: one-level vs two-level k-means on 2-D synthetic data of
# 100k / 250k / 500k points, 500 per cluster; Table 3: the 500k case at compression 5, 10, 15,
# 20), on a Tesla C2075 GPU against a Xeon E5-1410 CPU, units unlabelled (seconds, presumably).
PAPER_TABLE2 = {100000: (2.328, 2.78), 250000: (25.6, 4.96), 500000: (156.8, 6.2)}
PAPER_TABLE3 = {5: 6.2, 10: 5.76, 15: 4.83, 20: None}
TABLES_N_SUB = 1000          # subcluster size N; compression c gives N / c local centers


def main_tables(args):
    """Tables 2 and 3 re-shaped for this GPU: for n in {100k, 250k, 500k} 2-D points, 500 per
    blob, k = n / 500: one-level Lloyd on all points (a batch of one instance) against the
    two-level method at compression c = N / local_k in {5, 10, 15, 20} with N = 1000; 25
    Lloyd iterations, seeded init, every run graph-recorded and timed with CUDA events on
    its stream.  Reports times, speedups and each run's SSE over all scaled points; the
    oracle's times for the 100k case when host timing is on.  Context, not a driver line."""
    import numpy as np
    import torch

    import oracle
    from paper_1412_1947_gb300 import binding as B

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    iters, seed = 25, 1947
    ctx = B.pscl_ctx_create(0, 0, stream.cuda_stream)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b_.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b_))
        return statistics.median(ms)

    rows = []
    for n in (100000, 250000, 500000):
        k = n // 500
        raw = synth.blob_points(n // 500, 500, 2, seed=synth.BASE_SEED + 10 + n // 50000)
        x_dev = torch.from_numpy(raw).to(dev)
        one = B.Batch(x_dev, np.array([n], np.int64), [k], ctx=ctx)
        one_ms = timed(lambda: one.run(iters, seed, B.PSCL_PREC_FP32), args.steps)
        _, _, sse1 = one.result(labels=False)
        one.close()
        row = {"n": n, "k": k, "one_level_ms": one_ms, "one_level_sse": float(sse1[0]),
               "one_level_evals": n * k * iters, "two_level": []}
        for c in (5, 10, 15, 20):
            lk = -(-TABLES_N_SUB // c)
            job = B.Job(x_dev, ctx=ctx)
            job.option(B.PSCL_OPT_GRAPH)
            ms = timed(lambda: job.run(TABLES_N_SUB, lk, k, iters, seed, B.PSCL_PREC_FP32), args.steps)
            _, _, sse2 = job.result(labels=False)
            job.close()
            row["two_level"].append({"compression": c, "N": TABLES_N_SUB, "local_k": lk, "ms": ms,
                                     "speedup": one_ms / ms, "sse": sse2, "sse_ratio": sse2 / float(sse1[0])})
        if n == 100000 and not args.no_cpu:
            xs, _, _ = oracle.scale(raw)
            t0 = time.perf_counter()
            oracle.lloyd_seeded(xs, k, iters, seed)
            t1 = time.perf_counter()
            oracle.two_level(raw, TABLES_N_SUB, TABLES_N_SUB // 5, k, iters, seed)
            t2 = time.perf_counter()
            row["oracle_s"] = {"one_level": t1 - t0, "two_level_c5": t2 - t1,
                               "cores": os.cpu_count(), "note": "float64 C oracle, OpenMP over subclusters"}
        rows.append(row)
        del x_dev
    B.pscl_ctx_destroy(ctx)
    r500 = rows[-1]["two_level"][0]
    line = {"metric": "two-level speedup over one-level Lloyd (500k points, compression 5)", "value": r500["speedup"],
            "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic (2-D, 500 points per blob)",
            "config": {"workload": "tables_2d_500perblob", "iters": iters, "N": TABLES_N_SUB,
                       "compression": "N / local_k"},
            "rows": rows,
            "paper": {"table2_s": {str(k_): v for k_, v in PAPER_TABLE2.items()},
                      "table3_s": {str(k_): v for k_, v in PAPER_TABLE3.items()},
                      "hardware": "Tesla C2075 (two-level), Xeon E5-1410 (one-level)"}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium", choices=["small", "medium", "large", "uneven", "serving", "tables"])
    ap.add_argument("--rows-per-thread", type=int, default=0, choices=[0, 1, 2],
                    help="float32 assignment: 0 default, 1 one row per thread, 2 eight rows (d <= 16)")
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-n-max", type=float, default=1e6,
                    help="largest n of the serving stream (n is log-uniform in [1e4, this]); 1e7 is the "
                         "stream's stated range, 1e6 keeps a run within a minute")
    ap.add_argument("--oracle-n", type=int, default=1 << 17)
    ap.add_argument("--n", type=int, default=0,
                    help="run the workload's recipe at n points (same N, k, iterations), e.g. for a "
                         "profiler capture of a small case; 0 = the workload's own n")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--prec", default="tc", choices=["fp32", "tf32", "bf16", "tf32x3", "bf16x3", "tc"],
                    help="arithmetic of the Lloyd assignment (tf32/bf16: tensor cores + float32 near-tie "
                         "recheck; tc: the split mode that serves the shape, TF32x3 else BF16x3; every mode "
                         "assigns exactly as fp32)")
    args = ap.parse_args()
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the job server has no reference arm"}))
        else:
            main_serving(args)
        return
    if args.workload == "tables":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the tables workload has no reference arm; "
                              "its oracle times are in the same line"}))
        else:
            main_tables(args)
        return
    if args.workload == "uneven":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the uneven batch has no reference arm; "
                              "its oracle is timed in the cpu_baseline of the same line"}))
        else:
            main_uneven(args)
        return
    w = {"small": synth.SMALL, "medium": synth.MEDIUM, "large": synth.LARGE}[args.workload]
    if args.n:
        w = synth.scaled_down(w, args.n)
    if args.impl == "reference":
        reference_arm(args, w)
    else:
        main_arm(args, w)


if __name__ == "__main__":
    main()
