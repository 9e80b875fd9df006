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
SM_MAX_MHZ_NOMINAL = 2070.0
FP32_LANES_PER_SM = 128
FP64_TFLOPS_NOMINAL = 1.25


def measured_peaks():
    try:
        with open(MEASURED_PEAKS) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def fp32_peak(torch, device, clocks):
    """FP32 FMA peak (TFLOP/s) of this GPU from its unit counts and clock: SMs
    read from the device properties, 128 FP32 lanes per SM, 2 flop per FMA, at
    the maximum SM clock (the measured peaks file, else the sampled clocks,
    else the nominal 2070 MHz)."""
    sms = int(torch.cuda.get_device_properties(device).multi_processor_count)
    mhz = measured_peaks().get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or SM_MAX_MHZ_NOMINAL
    peak = sms * FP32_LANES_PER_SM * 2 * float(mhz) * 1e6 / 1e12
    return peak, "FP32 FMA: %d SMs (device properties) x 128 lanes x 2 x %.0f MHz (derived)" % (sms, mhz)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "mixed_fast", "fp64"])
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the cpu_baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-clustered", action="store_true",
                   help="skip the clustered 64-theta object of the default grid line")
    p.add_argument("--launch", default=None, metavar="ROWS,STAGES,BUCKETS,CONCURRENT[,QUEUE[,PRIOR]]",
                   help="pin the launch configuration (mra_set_launch) instead of running the autotuner, "
                        "e.g. 64,1,0,1 (QUEUE 1: leaf buckets as persistent work queues; PRIOR 0/1/2/3: the "
                        "prior's ancestor blocks staged by occupancy, in one buffer, two, two blocks at a time)")
    p.add_argument("--workload", default="grid", choices=["grid", "clustered", "massive", "swaths", "modis18"],
                   help="grid: n=131,072, 1 theta per call (default); clustered: n=2,097,152 with 64 theta per "
                        "call; massive: n=47,185,920, 1 theta per call; swaths: n=2,439,827, J=2, M=14, "
                        "r=49, 1 theta per call; modis18: n=4,194,304, J=2, M=18, r=49, 1 theta per call")
    return p.parse_args()


def max_over_ranks(x, world):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def whole_job_rate(n_obs, theta_per_call, steps, seconds, world):
    """obs*evals/s of the whole job: every rank evaluates its own `steps` calls
    of `theta_per_call` theta on the same tree (no data exchange), in the
    slowest rank's time."""
    return world * n_obs * theta_per_call * steps / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOAD_INFO = {
    "grid": dict(desc="grid n=131072 M=7 J=4 r=32 (r_hat=30), 1 theta per call", per_call=1, data=DATA),
    "clustered": dict(desc="clustered n=2097152 M=9 J=4 r=32 (r_hat=30), 64 theta per call (4x4x4 log grid)",
                      per_call=64,
                      data="synthetic: 70% of n=2097152 in 8 Gaussian clusters (sd 0.03), 30% uniform; z from an "
                           "exponential GP (sigma2=1, beta=0.05, tau2=0.01) by circulant embedding, seed 1908"),
    "massive": dict(desc="massive n=47185920 M=12 J=4 r=16, 1 theta per call", per_call=1,
                    data="synthetic: n=47185920 uniform on [0,1]^2 minus 200 discs (5% of the area); z from an "
                         "exponential GP (sigma2=1, beta=0.02, tau2=0.01) by circulant embedding, seed 1911"),
    "swaths": dict(desc="swaths n=2439827 M=14 J=2 r=49 (27 device levels), 1 theta per call", per_call=1,
                   data="synthetic: n=2439827 uniform on [0,1]^2 in slanted bands (80% coverage, straight gaps); "
                        "z from an exponential GP (sigma2=1, beta=0.05, tau2=0.01) by circulant embedding, "
                        "seed 1912"),
    "modis18": dict(desc="modis18 n=4194304 M=18 J=2 r=49 (35 device levels), 1 theta per call", per_call=1,
                    data="synthetic: n=4194304 uniform on [0,1]^2 in slanted bands (80% coverage, straight gaps); "
                         "z from an exponential GP (sigma2=1, beta=0.05, tau2=0.01) by circulant embedding, "
                         "seed 1913"),
}


def workload(name="grid"):
    from paper_1905_00141_gb300 import synth
    return synth.make(name)


def step_thetas(name):
    """theta of each timed call, [calls][per_call][3]"""
    if name == "clustered":
        from paper_1905_00141_gb300 import synth
        return synth.theta_grid_4x4x4()[None, :, :]
    if name == "massive":
        return np.array([[1.0, 0.02, 0.01], [1.2, 0.025, 0.012], [0.8, 0.016, 0.008], [1.1, 0.022, 0.009]])[:, None]
    return THETAS[:, None, :]


def config(precision, name="grid", d=None):
    info = WORKLOAD_INFO[name]
    c = {"workload": info["desc"], "n": int(len(d["x"])) if d is not None else None,
         "M": d["M"] if d is not None else None, "J": d["J"] if d is not None else None,
         "r": d["r"] if d is not None else None,
         "theta_per_call": info["per_call"], "precision": precision,
         "l2": "flushed between steps (256 MB write, outside the timed events)"}
    return c


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
    for f in ("mra_kernels.cuh", "mra_launch.cuh", "mra_bigleaf.cuh", "mra_predict.cuh", "mra_gram_tc.cuh",
              "mra_leafbasis_tc.cuh", "tc_sm100.cuh", "ff_math.h", "mra_internal.h"):
        with open(os.path.join(ROOT, "paper_1905_00141_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_counters(family, precision, key="bytes_per_launch"):
    """A per-family figure from the committed ncu captures (profiles/
    dram_traffic.json): DRAM bytes per launch, or the fraction of issue slots
    busy; None when the capture is of another precision or of kernel source
    that has changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if precision != "mixed" or t.get("csrc_sha256_prefix") != kernel_source_hash():
        return None
    return t.get(key, {}).get(family)


def measured_traffic(family, precision):
    return measured_counters(family, precision)


def clocks_rejected(c):
    if not c:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c["reasons"]):
        return True
    return c["sm_mhz"] < 0.6 * c["sm_max_mhz"] and "sw_power_cap" not in c["reasons"]


# ---------------------------------------------------------------- oracle arm --
def oracle_rate(d, seconds, max_evals=30, min_evals=1, name="grid", warm=True):
    """Time the FP64 CPU oracle, as it stands, on full evaluations of the workload."""
    import oracle
    oracle.build()
    t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    cores = oracle.max_threads()
    if warm:
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
                sample="%d full evaluations of the %s workload (n=%d) on %d host threads, %.1f s" %
                (done, name, n, cores, dt), seconds=dt, evals=done)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "massive":
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 CPU oracle is not run on the 47M-observation "
                          "tree (about 5 TFLOP and tens of GB of host memory per evaluation)"}), flush=True)
        return 0
    if args.workload in ("swaths", "modis18"):
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 CPU oracle takes minutes per evaluation of "
                          "the r=49 %s tree; its stored values are checked in tests/test_zv_%s_gpu.py" %
                          (args.workload, args.workload)}), flush=True)
        return 0
    d = workload(args.workload)
    thetas = step_thetas(args.workload).reshape(-1, 3)
    import oracle
    oracle.build()
    t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    for k in range(args.warmup if args.workload == "grid" else 0):
        t.loglik(thetas[k % len(thetas)])
    t0 = time.perf_counter()
    for k in range(args.steps):
        t.loglik(thetas[k % len(thetas)])
    dt = time.perf_counter() - t0
    n = t.n_used
    cores = oracle.max_threads()
    value = n * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": WORKLOAD_INFO[args.workload]["data"], "config": config("fp64", args.workload, d),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d full evaluations (one theta each) of the %s workload on %d host threads" %
                             (args.steps, args.workload, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm --
def timed_steps(g, torch, th_dev, out_dev, flush, stream, K):
    """K device-resident calls, each bracketed by CUDA events on `stream`;
    th_dev[c] holds the theta of call c (cycled), out_dev[c] its loglik."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    C = th_dev.shape[0]
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            g.loglik_device(th_dev[k % C].data_ptr(), th_dev.shape[1], out_dev[k % C].data_ptr(), 0,
                            stream.cuda_stream)
            ev[k][1].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def measure_precision(g, torch, precision, args, thetas, stream, flush, local):
    g.set_precision(precision)
    th_dev = torch.tensor(thetas, dtype=torch.float64, device="cuda").contiguous()
    out_dev = torch.zeros(thetas.shape[:2], dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        timed_steps(g, torch, th_dev, out_dev, flush, stream, thetas.shape[0])
    # timed region: the passes replay from captured CUDA graphs
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
    ms = timed_steps(g, torch, th_dev, out_dev, flush, stream, args.steps)
    clocks = sampler.stop() if not args.no_clocks else None
    ll = out_dev.cpu().numpy()
    # per-kernel times from a separate run of the same steps with kernel events
    g.profile(True)
    g.profile_read()
    timed_steps(g, torch, th_dev, out_dev, flush, stream, args.steps)
    prof = g.profile_read()
    g.profile(False)
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
    name = args.workload
    d = workload(name)
    thetas = step_thetas(name)
    per_call = thetas.shape[1]
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], device=local, precision=args.precision)
    st = g.stats()
    n = st["n_used"]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_measure(prec, a):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms, clocks, prof, ll = measure_precision(g, torch, prec, a, thetas, stream, flush, local)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return ms, clocks, prof, ll

    # launch configuration chosen by the library's autotuner (outside the timed region), or pinned
    def choose_launch():
        if args.launch:
            keys = ("leafbasis_rows", "leafbasis_stages", "bucket_set", "concurrent", "leaf_queue", "prior_stages")
            cfg = dict(zip(keys, (int(v) for v in args.launch.split(","))))
            g.set_launch(**cfg)
            return dict(cfg, pinned=True)
        return g.autotune(thetas[0][0], reps=3)

    tune = choose_launch()
    ms, clocks, prof, ll = one_measure(args.precision, args)
    attempt = 1
    if clocks_rejected(clocks):
        # the clock record of the timed region was rejected: measure once more
        ms, clocks, prof, ll = one_measure(args.precision, args)
        attempt = 2
    if clocks is not None:
        clocks["attempt"] = attempt
    t_total = max_over_ranks(sum(ms) / 1e3, world)
    value = whole_job_rate(n, per_call, args.steps, t_total, world)

    # the other precision on the same theta, for the mixed-vs-FP64 comparison
    other = "fp64" if args.precision != "fp64" else "mixed"
    other_line, ll_o = None, None
    if name not in ("massive", "swaths", "modis18"):
        oargs = argparse.Namespace(**vars(args))
        if name != "grid":
            oargs.steps, oargs.warmup = min(args.steps, 2), 1
        ms_o, _, prof_o, ll_o = one_measure(other, oargs)
        other_line = {"precision": other, "value": world * n * per_call * oargs.steps / (sum(ms_o) / 1e3),
                      "ms_per_step": sum(ms_o) / oargs.steps, "steps": oargs.steps}
        g.set_precision(args.precision)
        choose_launch()
    # the fast mixed mode (FP32 remainder recursions) on the same steps
    fast_line, ll_f = None, None
    if args.precision == "mixed" and name == "grid":
        g.set_precision("mixed_fast")
        choose_launch()
        ms_f, _, _, ll_f = one_measure("mixed_fast", args)
        fast_line = {"precision": "mixed_fast", "value": whole_job_rate(n, per_call, args.steps, sum(ms_f) / 1e3, 1),
                     "ms_per_step": sum(ms_f) / args.steps}
        g.set_precision(args.precision)
        choose_launch()

    # end to end: host theta (pinned) in, host loglik out, through mra_loglik
    th_host = torch.tensor(thetas, dtype=torch.float64).pin_memory().numpy()
    C = th_host.shape[0]
    for k in range(args.warmup):
        g.loglik(th_host[k % C])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        g.loglik(th_host[k % C])
    e2e_dt = time.perf_counter() - t0
    e2e_value = whole_job_rate(n, per_call, args.steps, max_over_ranks(e2e_dt, world), world)

    if rank != 0:
        if world > 1:
            dist.barrier()
        return 0

    # accuracy: against the FP64 oracle (grid), against the FP64 GPU path
    # (clustered); not measured at the 47M size (sampled leaves are in the tests)
    import oracle
    oracle.build()
    if name == "grid":
        ot = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
        ref, _ = ot.loglik(thetas.reshape(-1, 3))
        ot.close()
        ref = ref.reshape(thetas.shape[:2])
        acc = {"against": "FP64 CPU oracle", args.precision: float(np.max(np.abs(ll - ref)) / n),
               other: float(np.max(np.abs(ll_o - ref)) / n)}
        if ll_f is not None:
            acc["mixed_fast"] = float(np.max(np.abs(ll_f - ref)) / n)
    elif ll_o is not None:
        acc = {"against": "FP64 GPU path", args.precision: float(np.max(np.abs(ll - ll_o)) / n)}
    elif name in ("swaths", "modis18"):
        acc = stored_accuracy(name, d, thetas, ll, n, args.precision)
    else:
        acc = {"against": None, "note": "FP64 does not fit one theta of this tree; sampled leaves against the "
                                        "oracle in tests/test_zx_massive_gpu.py"}

    # roofline of the dominant kernel family
    fam = max(prof, key=lambda k: prof[k][1])
    launches, fam_ms = prof[fam]
    fl_per_launch = st["flops_by_kernel"][fam] * per_call * args.steps / launches
    achieved = fl_per_launch / (fam_ms / launches / 1e3) / 1e12
    if args.precision != "fp64":
        peak, peak_note = fp32_peak(torch, local, clocks)
    else:
        peak = FP64_TFLOPS_NOMINAL
        peak_note = "FP64: nominal 1.25 TFLOP/s (recipe)"
    roof = {"bound": "alu", "kernel": fam, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": measured_traffic(fam, args.precision) if name == "grid" else None,
            "peak_source": peak_note, "launch_ms": fam_ms / launches, "flops_per_launch": fl_per_launch,
            "issue_active_frac_ncu": measured_counters(fam, args.precision, "issue_active_frac")
            if name == "grid" else None}
    roof["families"] = family_fractions(prof, st, per_call, args.steps, peak, args.precision, name)

    cpu = None
    if not args.no_cpu_baseline:
        if name == "grid":
            cpu = oracle_rate(d, args.cpu_seconds)
        elif name == "clustered":
            cpu = oracle_rate(d, args.cpu_seconds, max_evals=1, name=name, warm=False)
        elif name == "massive":
            cpu = {"value": None, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                   "sample": "not run: about 5 TFLOP per evaluation of the 47M tree"}
        else:
            cpu = {"value": None, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                   "sample": "not run: one evaluation of this r=49 tree took the oracle 9 to 23 minutes on 8 "
                             "host threads (the stored values' timings)"}
        if cpu:
            cpu.pop("seconds", None)
            cpu.pop("evals", None)

    # the same steps with the leaf Gram on the tensor cores (exact BF16 slices)
    gram_tc = None
    if name == "grid" and args.precision == "mixed":
        cfg = {k: tune[k] for k in ("leafbasis_rows", "leafbasis_stages", "bucket_set", "concurrent", "leaf_queue",
                                    "prior_stages") if k in tune}
        g.set_launch(**cfg, gram_tensor_cores=True)
        ms_t, _, prof_t, ll_t = measure_precision(g, torch, args.precision, args, thetas, stream, flush, local)
        g.set_launch(**cfg, gram_tensor_cores=False)
        gram_tc = {"ms_per_step": sum(ms_t) / args.steps, "value": whole_job_rate(n, per_call, args.steps,
                                                                                 sum(ms_t) / 1e3, 1),
                   "leafgram_ms_per_step": prof_t.get("leafgram", (0, 0.0))[1] / args.steps,
                   "accuracy_abs_dl_per_n": float(np.max(np.abs(ll_t - ref)) / n),
                   "note": "the same timed steps with mra_tune_t.gram_tensor_cores = 1 (tcgen05 BF16 MMAs of exact "
                           "fixed-grid slices; column exponents by k_gram_colexp); accuracy against the FP64 CPU oracle"}
    # the same steps with the leaf basis's remainder products on the tensor cores
    lb_tc = None
    if name == "grid" and args.precision == "mixed":
        g.set_launch(**cfg, leafbasis_tensor_cores=True)
        ms_l, _, prof_l, ll_l = measure_precision(g, torch, args.precision, args, thetas, stream, flush, local)
        g.set_launch(**cfg, leafbasis_tensor_cores=False)
        lb_launches, lb_ms = prof_l.get("leafbasis", (0, 0.0))
        lb_tc = {"ms_per_step": sum(ms_l) / args.steps, "value": whole_job_rate(n, per_call, args.steps,
                                                                               sum(ms_l) / 1e3, 1),
                 "leafbasis_ms_per_step": lb_ms / args.steps,
                 "leafbasis_alu_tflops": (st["flops_by_kernel"]["leafbasis"] * per_call * args.steps / lb_ms / 1e9
                                          if lb_ms > 0 else None),
                 "accuracy_abs_dl_per_n": float(np.max(np.abs(ll_l - ref)) / n),
                 "note": "the same timed steps with mra_tune_t.leafbasis_tensor_cores = 1 (remainder products as "
                         "tcgen05 BF16 MMAs of five exact fixed-grid slices per value, 128 rows per CTA); accuracy "
                         "against the FP64 CPU oracle"}
    pred = prediction_line(g, d, args.precision) if name == "grid" else None
    clus = None
    if name == "grid" and args.precision == "mixed" and not args.no_clustered:
        g.close()
        clus = clustered_line(torch, stream, flush, local)

    step_ms = 1e3 * t_total / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+ff",
        "data": WORKLOAD_INFO[name]["data"], "config": config(args.precision, name, d),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * per_call,
                "d2h_bytes_per_step": 12 * per_call},
        "gpu_launches": int(st["launches_per_pass"]) * args.steps if st["launches_per_pass"] else
        int(sum(v[0] for v in prof.values())),
        "clocks": clocks,
        "accuracy_abs_dl_per_n": acc,
        "other_precision": other_line,
        "fast_mixed": fast_line,
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "flops_per_eval": st["flops_per_theta"],
        "launch_config": {k: tune[k] for k in ("leafbasis_rows", "leafbasis_stages", "bucket_set", "concurrent",
                                                "gram_tensor_cores", "leaf_queue", "prior_stages", "pinned")
                          if k in tune},
        "gram_tensor_cores": gram_tc,
        "leafbasis_tensor_cores": lb_tc,
        "predict": pred,
        "clustered": clus,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
    g.close()
    return 0


def stored_accuracy(name, d, thetas, ll, n, precision):
    """|dl|/n of the timed calls whose theta has a stored FP64 CPU oracle
    value (tests/golden/full_size_oracle.txt, used only when this draw of the
    workload matches the value's fingerprint); the FP64 kernels do not fit
    these depths."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        from golden_values import fingerprint_matches, golden
    finally:
        sys.path.pop(0)
    rows = golden(name)
    th = thetas.reshape(-1, 3)
    vals = np.asarray(ll).reshape(-1)
    errs = []
    for r in rows:
        if not fingerprint_matches(d, r[3]):
            continue
        for k in range(th.shape[0]):
            if np.allclose(th[k], r[0], rtol=1e-12, atol=0):
                errs.append(abs(vals[k] - r[1]) / n)
    if not errs:
        return {"against": None, "note": "no stored oracle value matches these calls; the FP64 kernels do not "
                                         "fit this depth"}
    return {"against": "FP64 CPU oracle (stored values)", "calls_checked": len(errs), precision: float(max(errs))}


def family_fractions(prof, st, per_call, steps, alu_peak, precision, name):
    """Every kernel family's place against its two roofs: the ALU roof
    (algorithmic flops per launch from mra_stats over the live mean launch
    time, against the FP32 FMA or FP64 peak) and the HBM roof (DRAM bytes per
    launch of the committed ncu capture, while the kernel source matches it,
    over the same time, against the measured copy bandwidth)."""
    hbm = measured_peaks().get("hbm_gbs")
    out = {}
    for fam, (launches, ms) in prof.items():
        t = ms / launches / 1e3
        fl = st["flops_by_kernel"].get(fam, 0.0) * per_call * steps / launches
        e = {"launches_per_step": launches / steps, "ms_per_launch": 1e3 * t,
             "alu_tflops": fl / t / 1e12, "alu_frac": fl / t / 1e12 / alu_peak}
        b = measured_traffic(fam, precision) if name == "grid" else None
        if b is not None and hbm:
            # the committed traffic is per launch of the captured configuration
            e["hbm_gbs"] = b / t / 1e9
            e["hbm_frac"] = b / t / 1e9 / hbm
        out[fam] = e
    return out


def clustered_line(torch, stream, flush, local, precision="mixed", calls=2, warm=1):
    """The batched uneven workload as the benchmark's second line of work: the
    clustered tree (n = 2,097,152, M = 9, J = 4, r = 32), 64 theta (the 4x4x4
    log grid) per call, inputs resident, CUDA events on the call's stream, L2
    flushed between calls.  Accuracy against the FP64 CPU oracle's stored values
    at four of the 64 theta (tests/golden/full_size_oracle.txt, used when this
    machine's draw of the data matches their fingerprint), and the FP64 GPU
    path timed on those four theta for the mixed-vs-FP64 ratio."""
    from paper_1905_00141_gb300 import mra, synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        from golden_values import fingerprint_matches, golden
    finally:
        sys.path.pop(0)
    d = synth.clustered()
    grid = synth.theta_grid_4x4x4()
    rows0 = golden("clustered")
    for r in rows0:
        k = int(np.argmin(np.abs(grid - r[0]).sum(axis=1)))
        if np.allclose(grid[k], r[0], rtol=1e-12, atol=0):
            grid[k] = r[0]
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], device=local, precision=precision)
    try:
        n = g.stats()["n_used"]
        g.set_launch(64, 1, 0, True)
        th_dev = torch.tensor(grid[None], dtype=torch.float64, device="cuda").contiguous()
        out_dev = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
        for _ in range(warm):
            timed_steps(g, torch, th_dev, out_dev, flush, stream, 1)
        ms = timed_steps(g, torch, th_dev, out_dev, flush, stream, calls)
        ll = out_dev.cpu().numpy()[0]
        # the leaf buckets as persistent work queues (largest leaf first), same calls
        g.set_launch(64, 1, 0, True, leaf_queue=True)
        timed_steps(g, torch, th_dev, out_dev, flush, stream, 1)
        ms_q = timed_steps(g, torch, th_dev, out_dev, flush, stream, calls)
        same_q = bool(np.array_equal(out_dev.cpu().numpy()[0], ll))
        g.set_launch(64, 1, 0, True)
        g.profile(True)
        g.profile_read()
        timed_steps(g, torch, th_dev, out_dev, flush, stream, 1)
        prof = g.profile_read()
        g.profile(False)
        rows = golden("clustered")
        acc = None
        pick = []
        if rows and all(fingerprint_matches(d, r[3]) for r in rows):
            # the stored theta sit in their slots of the grid up to the last bits
            # of the platform's libm; the accuracy call uses the stored values
            pick = [int(np.argmin(np.abs(grid - r[0]).sum(axis=1))) for r in rows]
            ref = np.array([r[1] for r in rows])
            acc = {"against": "FP64 CPU oracle (stored values)", "theta_index": pick,
                   precision: float(np.max(np.abs(ll[pick] - ref)) / n)}
        # the FP64 GPU path on four theta of the grid
        four = grid[pick] if pick else grid[[0, 21, 42, 60]]
        g.set_precision("fp64")
        th4 = torch.tensor(four[None], dtype=torch.float64, device="cuda").contiguous()
        o4 = torch.zeros((1, len(four)), dtype=torch.float64, device="cuda")
        timed_steps(g, torch, th4, o4, flush, stream, 1)
        ms64 = timed_steps(g, torch, th4, o4, flush, stream, 1)
        ll64 = o4.cpu().numpy()[0]
        if acc is not None:
            acc["fp64"] = float(np.max(np.abs(ll64 - ref)) / n)
        t = sum(ms) / 1e3
        per_theta_ms = 1e3 * t / (calls * 64)
        fp64_per_theta_ms = ms64[0] / len(four)
        return {"workload": WORKLOAD_INFO["clustered"]["desc"], "n": n, "precision": precision,
                "value": n * 64 * calls / t, "unit": UNIT, "calls": calls, "warmup_calls": warm,
                "ms_per_step": 1e3 * t / calls, "ms_per_theta": per_theta_ms,
                "launch_config": {"leafbasis_rows": 64, "leafbasis_stages": 1, "bucket_set": 0, "concurrent": 1,
                                  "pinned": True},
                "fp64_ms_per_theta": fp64_per_theta_ms, "mixed_vs_fp64": fp64_per_theta_ms / per_theta_ms,
                "leaf_queue": {"ms_per_theta": sum(ms_q) / (calls * 64), "same_loglik_bits": same_q,
                               "note": "the same calls with each leaf bucket as a persistent work-queue kernel"},
                "accuracy_abs_dl_per_n": acc,
                "kernels_ms_per_step": {k: v[1] for k, v in prof.items()},
                "l2": "flushed between calls (256 MB write, outside the timed events)"}
    finally:
        g.close()


def prediction_line(g, d, precision, npts=131072, reps=3):
    """Posterior prediction (mra_predict) at npts random points of the
    workload's domain: host-API wall time per call (one likelihood pass that
    keeps the factors, the top-down pass, the basis at the points, one warp
    per point, transfers included), the largest difference from the other
    precision, and two points against the oracle's likelihood differences."""
    import oracle
    x, y = d["x"], d["y"]
    rng = np.random.default_rng(1905)
    px = rng.uniform(x.min(), x.max(), npts)
    py = rng.uniform(y.min(), y.max(), npts)
    th = [1.0, 0.05, 0.01]
    g.predict(th, px[:1024], py[:1024])
    # cold: a new theta every call (the likelihood pass that keeps the factors
    # runs each time); warm: the same theta again (the kept factors are reused)
    t0 = time.perf_counter()
    for k in range(reps):
        m, v = g.predict([th[0] * (1.0 + 0.01 * (k + 1)), th[1], th[2]], px, py)
    dt_cold = (time.perf_counter() - t0) / reps
    m, v = g.predict(th, px, py)
    t0 = time.perf_counter()
    for _ in range(reps):
        m, v = g.predict(th, px, py)
    dt = (time.perf_counter() - t0) / reps
    other = "fp64" if precision != "fp64" else "mixed"
    g.set_precision(other)
    mo, vo = g.predict(th, px[:4096], py[:4096])
    g.set_precision(precision)
    chk = []
    for k in range(2):
        a, b = float(px[k]), float(py[k])
        if x.min() < a < x.max() and y.min() < b < y.max():
            rm, rv = oracle.predict_by_loglik(x, y, d["z"], d["M"], d["J"], d["r"], th, a, b)
            chk.append((abs(m[k] - rm), abs(v[k] - rv)))
    return {"points": npts, "theta": th, "ms_per_call": 1e3 * dt_cold, "points_per_s": npts / dt_cold,
            "ms_per_call_same_theta": 1e3 * dt, "points_per_s_same_theta": npts / dt,
            "timing": "host API wall time, transfers included; a new theta per call (the likelihood pass that "
                      "keeps the factors included), and the same theta again (the kept factors reused)",
            "max_abs_diff_vs_" + other: float(max(np.max(np.abs(m[:4096] - mo)), np.max(np.abs(v[:4096] - vo)))),
            "oracle_check": {"points": len(chk), "route": "likelihood differences of the FP64 CPU oracle",
                             "max_abs_err_mean": float(max(c[0] for c in chk)) if chk else None,
                             "max_abs_err_var": float(max(c[1] for c in chk)) if chk else None}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
