#!/usr/bin/env python3
"""Throughput of the f-thermostat hot path on GB300: GLE replica-steps per second.

Workload (one GPU): dense SPD M, N = 4096, M = Q diag(lam) Q^T with Q Haar and lam
log-uniform in [1, 1e3] (seeded), f = Fermi(beta = 5, mu = median lam), GLE with s = 4
fitted on the host, dt = 0.1 / sqrt(1e3), R = 256 replicas, FP32 state, force GEMM in
the chosen precision, every element of <p p^T> accumulated (FP32 block partials, FP64
block sums).  One step = force, B, O, sample + accumulate, O, B, A over all replicas.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank runs its own replicas of the
same matrix (replicas are independent: weak scaling, no collective in the timed region).
"""
from __future__ import annotations

import argparse
import json
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

import fth_synth as syn  # noqa: E402

N, LAM, R, BETA = 4096, (1.0, 1000.0), 256, 5.0
SEED = syn.BASE_SEED + 1
BLOCK = 1000
METRIC, UNIT = "GLE replica-steps/s", "replica-steps/s"
WORKLOAD = "dense SPD N=4096, lambda log-uniform [1,1e3], Fermi beta=5 mu=median, R=256, all elements"
L2_BYTES = 129 * 2 ** 20
CPU_SAMPLE_REPLICAS = 16
CPU_BUDGET_S = 15.0
REF_BUDGET_S = 90.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _workload():
    M, lam, _ = syn.dense_spd(N, LAM[0], LAM[1], seed=SEED)
    mu = float(np.median(lam))
    from paper_1402_2095_gb300 import fit
    a_p, c_p, dt, rep = fit.load_gle("fermi_b5_1_1000")
    return M, lam, mu, a_p, c_p, dt, rep


# ---------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="fth_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if f[5 + k].lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------- roofline
def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu capture of this kernel, or None when
    the kernel's source has changed since the capture (hash mismatch)."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) == 4 and f[0] == kernel:
            try:
                src = open(os.path.join(ROOT, f[1]), "rb").read()
            except OSError:
                return None
            if hashlib.sha256(src).hexdigest()[:16] == f[2]:
                return int(f[3])
    return None


def roofline(prof, precision, n, R, stack_cols, peaks, peak_kind):
    """Dominant kernel (largest device time) against its bound."""
    name, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_s = ms / cnt / 1e3
    tf32_ratio = 1.1 / 2.25           # nominal dense TF32 / BF16 tensor rate
    sustained = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    fp32_alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if name == "force_tc":
        flops = 2.0 * n * n * R
        peak = sustained * (tf32_ratio if precision == "tf32" else 1.0)
        out = {"bound": "tensor", "unit": "TFLOP/s", "achieved": flops / per_launch_s / 1e12,
               "peak": peak}
    elif name == "syrk_tc":
        flops = float(n) * (n + 1) * stack_cols
        out = {"bound": "tensor", "unit": "TFLOP/s", "achieved": flops / per_launch_s / 1e12,
               "peak": sustained * tf32_ratio}
    elif name in ("force_fp32", "syrk_fp32"):
        flops = 2.0 * n * n * R if name == "force_fp32" else float(n) * (n + 1) * stack_cols
        out = {"bound": "alu", "unit": "TFLOP/s", "achieved": flops / per_launch_s / 1e12,
               "peak": fp32_alu}
    else:   # gle_dense: HBM bytes per element
        op_bytes = {"tf32": 4, "bf16x3": 4, "fp32": 0}[precision]
        byts = (28 + 24 + 4 + op_bytes) * n * R
        out = {"bound": "hbm", "unit": "GB/s", "achieved": byts / per_launch_s / 1e9,
               "peak": peaks["hbm_gbs"]}
    out["frac"] = out["achieved"] / out["peak"]
    out["kernel"] = name
    out["launch_us"] = per_launch_s * 1e6
    out["peak_source"] = f"{peak_kind} ({'sustained' if out['bound'] == 'tensor' else 'copy'})"
    out["traffic"] = _traffic(name)
    out["share"] = {k: round(v[0] / sum(x[0] for x in prof.values()), 4) for k, v in prof.items()}
    return out


# ---------------------------------------------------------------------- CPU oracle
def cpu_baseline(M, a_p, c_p, dt, budget_s=CPU_BUDGET_S, replicas=CPU_SAMPLE_REPLICAS):
    """The FP64 oracle as it stands on the host cores, on the same matrix and GLE with
    a replica sample, every element accumulated; timed for about budget_s."""
    from oracle.fth import OracleFTH
    pairs = syn.upper_pairs(M.shape[0])
    o = OracleFTH(M=M.astype(np.float32).astype(np.float64), a_p=a_p, c_p=c_p, dt=dt,
                  replicas=replicas, seed=SEED, block=BLOCK, pairs=pairs)
    o.run(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.run(1)
        steps += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": replicas * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"N={M.shape[0]}, {replicas} replicas, all {len(pairs)} elements, "
                      f"{steps} steps in {el:.1f} s"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    M, lam, mu, a_p, c_p, dt, rep = _workload()
    from oracle.fth import OracleFTH
    pairs = syn.upper_pairs(N)
    o = OracleFTH(M=M.astype(np.float32).astype(np.float64), a_p=a_p, c_p=c_p, dt=dt,
                  replicas=CPU_SAMPLE_REPLICAS, seed=SEED, block=BLOCK, pairs=pairs)
    o.run(min(max(args.warmup, 1), 2))
    # each step is a bounded sample (CPU_SAMPLE_REPLICAS of the R replicas, all
    # elements); the run stops after REF_BUDGET_S if K steps would take longer
    steps, t0 = 0, time.perf_counter()
    while steps < args.steps and time.perf_counter() - t0 < REF_BUDGET_S:
        o.run(1)
        steps += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = CPU_SAMPLE_REPLICAS * steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": el / max(steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "replicas_sampled": CPU_SAMPLE_REPLICAS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"N={N}, {CPU_SAMPLE_REPLICAS} of {R} replicas per step, "
                                   f"all {len(pairs)} elements, {steps} steps in {el:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_1402_2095_gb300 import FTH, build
    build.build()
    M, lam, mu, a_p, c_p, dt, rep = _workload()
    M32 = M.astype(np.float32)
    Md = torch.from_numpy(M32).cuda()
    stream = torch.cuda.current_stream()
    f = FTH(M=Md, a_p=a_p, c_p=c_p, dt=dt, replicas=R, seed=SEED + 7919 * rank,
            precision=args.precision, track="all", block=BLOCK, stream=stream)
    f.run(args.warmup)
    torch.cuda.synchronize()
    l0 = f.info()["launches"]

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    f.run(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    launches = f.info()["launches"] - l0
    f.poll()

    # per-kernel device time, CUDA events on the launching stream (separate pass)
    f.profile(True)
    f.run(min(args.steps, 2000))
    prof = f.profile_read()
    f.profile(False)
    peaks, peak_kind = _peaks()
    stack_cols = (2048 // R) * R
    roof = roofline(prof, args.precision, N, R, stack_cols, peaks, peak_kind)

    # end to end through the public API with host buffers: pinned M in, results out
    Mh = torch.from_numpy(M32).pin_memory()
    pairs = syn.upper_pairs(N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = FTH(M=Mh, a_p=a_p, c_p=c_p, dt=dt, replicas=R, seed=SEED + 7919 * rank + 1,
            precision=args.precision, track="all", block=BLOCK, stream=stream)
    g.run(args.steps)
    vals, errs = g.elements(pairs)
    t_e2e = time.perf_counter() - t0
    h2d = M32.nbytes + pairs.shape[0] * 8
    d2h = pairs.shape[0] * 3 * 8
    g.close()
    del g

    value = R * args.steps * world / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "replicas_per_gpu": R, "precision": args.precision,
                   "track": "all", "s": 4, "dt": dt, "block": BLOCK, "mu": mu,
                   "fit_max_rel_err": rep.get("max_rel_err"),
                   "l2": "per-step working set > L2: M %d MB + state %d MB + staged samples %d MB"
                         " + partial sums %d MB; steps back to back" % (
                             M32.nbytes >> 20, (8 * N * R * 4) >> 20, (N * stack_cols * 4) >> 20,
                             ((N // 128) * (N // 128 + 1) // 2 * 128 * 128 * 4) >> 20),
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "e2e": {"value": R * args.steps * world / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(M, a_p, c_p, dt)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
