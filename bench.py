#!/usr/bin/env python
"""MRA log-likelihood throughput on GB300: observations x evaluations per second.

One step = one full likelihood evaluation (prior build, leaf posterior, upward
pass, root) of the gridded workload (n=131,072 observations on a jittered
382x382 grid with 10% of the cells missing, M=7 levels, J=4, r=32 -> 30 knots
per region) at one theta, through the library's C ABI.  Inputs (the partition
and the observations) are resident on the device; each step's theta is read
from device memory and its loglik written to device memory.  The L2 cache is
flushed (a 256 MB write) between timed steps, outside the timed events.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the baseline arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MRA loglik obs·evals/sec, mixed vs FP64 on 1 GB300 at |Δℓ|/n≤1e-6; roofline %"
UNIT = "obs*evals/s"
WORKLOAD = "grid"
DATA = "synthetic: jittered 382x382 grid, 10% cells dropped, trimmed to n=131072; z from an exponential GP " \
       "(sigma2=1, beta=0.05, tau2=0.01) by circulant embedding, seed 1907"
# theta visited by the timed steps (a small cloud around the generating value, as an optimiser would)
THETAS = np.array([[1.0, 0.05, 0.01], [1.2, 0.06, 0.012], [0.8, 0.04, 0.008], [1.1, 0.055, 0.009]])
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FP64_TFLOPS_NOMINAL = 1.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the cpu_baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    from paper_1905_00141_gb300 import synth
    d = synth.grid()
    return d


def config(precision):
    return {"workload": "grid n=131072 M=7 J=4 r=32 (r_hat=30), 1 theta per call", "n": 131072, "M": 7, "J": 4,
            "r": 32, "r_hat": 30, "theta_per_call": 1, "precision": precision,
            "l2": "flushed between steps (256 MB write, outside the timed events)"}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), reasons=parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        active = sorted({names[i] for r in rows for i, v in enumerate(r["reasons"]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": active, "samples": len(rows)}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("mra_kernels.cuh", "mra_launch.cuh"):
        with open(os.path.join(ROOT, "paper_1905_00141_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(family, precision):
    """DRAM bytes per launch of a kernel family from the committed ncu launch
    list, or None when that capture is of another precision or of kernel
    source that has changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if precision != "mixed" or t.get("csrc_sha256_prefix") != kernel_source_hash():
        return None
    return t.get("bytes_per_launch", {}).get(family)


def clocks_rejected(c):
    if not c:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c["reasons"]):
        return True
    return c["sm_mhz"] < 0.6 * c["sm_max_mhz"] and "sw_power_cap" not in c["reasons"]


# ---------------------------------------------------------------- oracle arm --
def oracle_rate(d, seconds, max_evals=30, min_evals=1):
    """Time the FP64 CPU oracle, as it stands, on full evaluations of the workload."""
    import oracle
    oracle.build()
    t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    cores = oracle.max_threads()
    t.loglik(THETAS[0])  # warm caches / threads
    done = 0
    t0 = time.perf_counter()
    while done < min_evals or (time.perf_counter() - t0 < seconds and done < max_evals):
        t.loglik(THETAS[done % len(THETAS)])
        done += 1
    dt = time.perf_counter() - t0
    n = t.n_used
    t.close()
    return dict(value=n * done / dt, unit=UNIT, cores=cores, kind="oracle",
                sample="%d full evaluations of the grid workload (n=%d) on %d host threads, %.1f s" %
                (done, n, cores, dt), seconds=dt, evals=done)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    d = workload()
    import oracle
    oracle.build()
    t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    for k in range(args.warmup):
        t.loglik(THETAS[k % len(THETAS)])
    t0 = time.perf_counter()
    for k in range(args.steps):
        t.loglik(THETAS[k % len(THETAS)])
    dt = time.perf_counter() - t0
    n = t.n_used
    cores = oracle.max_threads()
    value = n * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA,
            "config": config("fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d full evaluations of the grid workload on %d host threads" %
                             (args.steps, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm --
def timed_steps(g, torch, th_dev, out_dev, flush, stream, K, n):
    """K device-resident steps, each bracketed by CUDA events on `stream`."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            g.loglik_device(th_dev[k % len(THETAS)].data_ptr(), 1, out_dev[k % len(THETAS)].data_ptr(), 0,
                            stream.cuda_stream)
            ev[k][1].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def measure_precision(g, torch, precision, args, d, stream, flush, local):
    g.set_precision(precision)
    th_dev = torch.tensor(THETAS, dtype=torch.float64, device="cuda")
    out_dev = torch.zeros(len(THETAS), dtype=torch.float64, device="cuda")
    th_rows = [th_dev[i:i + 1] for i in range(len(THETAS))]
    for _ in range(args.warmup):
        timed_steps(g, torch, th_rows, out_dev, flush, stream, len(THETAS), 0)
    g.profile(True)
    g.profile_read()
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
    ms = timed_steps(g, torch, th_rows, out_dev, flush, stream, args.steps, 0)
    clocks = sampler.stop() if not args.no_clocks else None
    prof = g.profile_read()
    g.profile(False)
    ll = out_dev.cpu().numpy()
    return ms, clocks, prof, ll


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_1905_00141_gb300 import build as mbuild
    from paper_1905_00141_gb300 import mra
    if rank == 0 or world == 1:
        mbuild.build()
    if world > 1:
        dist.barrier()
    d = workload()
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], device=local, precision=args.precision)
    st = g.stats()
    n = st["n_used"]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_measure(prec):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms, clocks, prof, ll = measure_precision(g, torch, prec, args, d, stream, flush, local)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return ms, clocks, prof, ll

    ms, clocks, prof, ll = one_measure(args.precision)
    if clocks_rejected(clocks):
        ms, clocks, prof, ll = one_measure(args.precision)
    t_total = sum(ms) / 1e3
    if world > 1:
        tt = torch.tensor([t_total], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt[0])
    value = world * n * args.steps / t_total

    # the other precision on the same steps, for the mixed-vs-FP64 comparison
    other = "fp64" if args.precision == "mixed" else "mixed"
    ms_o, _, prof_o, ll_o = one_measure(other)
    g.set_precision(args.precision)

    # end to end: host theta (pinned) in, host loglik out, through mra_loglik
    th_host = torch.tensor(THETAS, dtype=torch.float64).pin_memory().numpy()
    for k in range(args.warmup):
        g.loglik(th_host[k % len(THETAS)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        g.loglik(th_host[k % len(THETAS)])
    e2e_dt = time.perf_counter() - t0
    e2e_value = world * n * args.steps / e2e_dt if world == 1 else None
    if world > 1:
        tt = torch.tensor([e2e_dt], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_value = world * n * args.steps / float(tt[0])

    if rank != 0:
        if world > 1:
            dist.barrier()
        return 0

    # accuracy of both precisions against the FP64 oracle at the step thetas
    import oracle
    oracle.build()
    ot = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    ref, _ = ot.loglik(THETAS)
    ot.close()
    acc = {args.precision: float(np.max(np.abs(ll - ref)) / n), other: float(np.max(np.abs(ll_o - ref)) / n)}

    # roofline of the dominant kernel family
    fam = max(prof, key=lambda k: prof[k][1])
    launches, fam_ms = prof[fam]
    fl_per_launch = st["flops_by_kernel"][fam] * args.steps / launches
    achieved = fl_per_launch / (fam_ms / launches / 1e3) / 1e12
    if args.precision == "mixed":
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        peak_note = "FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz (derived, no tensor cores on this path)"
    else:
        peak = FP64_TFLOPS_NOMINAL
        peak_note = "FP64: nominal 1.25 TFLOP/s (recipe)"
    roof = {"bound": "alu", "kernel": fam, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": measured_traffic(fam, args.precision), "peak_source": peak_note,
            "launch_ms": fam_ms / launches, "flops_per_launch": fl_per_launch}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_rate(d, args.cpu_seconds)
        cpu.pop("seconds", None)
        cpu.pop("evals", None)

    step_ms = 1e3 * t_total / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": DATA,
        "config": config(args.precision),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24, "d2h_bytes_per_step": 12},
        "gpu_launches": int(st["launches_per_pass"]) * args.steps if st["launches_per_pass"] else
        int(sum(v[0] for v in prof.values())),
        "clocks": clocks,
        "accuracy_abs_dl_per_n": acc,
        "other_precision": {"precision": other, "value": world * n * args.steps / (sum(ms_o) / 1e3),
                            "ms_per_step": sum(ms_o) / args.steps},
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "flops_per_eval": st["flops_per_theta"],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
    g.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
