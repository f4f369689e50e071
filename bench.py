#!/usr/bin/env python3
"""Throughput of the f-thermostat hot path on GB300: GLE replica-steps per second.

Default workload (one GPU): dense SPD M, N = 4096, M = Q diag(lam) Q^T with Q Haar and
lam log-uniform in [1, 1e3] (seeded), f = Fermi(beta = 5, mu = median lam), GLE with
s = 4 fitted on the host, dt = 0.1 / sqrt(1e3), R = 256 replicas, FP32 state, force
GEMM in the chosen precision (TF32 by default), every element of <p p^T> accumulated
(FP32 block partials, FP64 block sums).  One step = force, B, O, sample + accumulate,
O, B, A over all replicas.

Other workloads (--workload): small_fp64 (N = 32 dense FP64, R = 16, all elements),
lattice64 (64^3 periodic lattice, CSR FP32, R = 64, diagonal + nearest-neighbour
elements) and ragged512 (512 dense problems of ragged order in one problem pool).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload dense4096|small_fp64|lattice64|ragged512]
                       [--precision ...]
Prints one JSON line (rank 0).  Under torchrun each rank runs its own slice of replicas
(replica_offset = rank * R, same seed): weak scaling, no collective in the timed region.
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

METRIC, UNIT = "GLE replica-steps/s", "replica-steps/s"
# arithmetic of the force contraction (FP32 accumulation everywhere but fp64)
DTYPE = {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3", "fp64": "f64"}
# the end-to-end pass runs at least this many steps (more when --steps asks for more), so
# the context creation, the matrix upload and the element read-out weigh as in a run of
# useful length rather than dominating a short timed loop
E2E_MIN_STEPS = 10000
CPU_BUDGET_S = 15.0
REF_BUDGET_S = 90.0


# ---------------------------------------------------------------------- workloads
class Workload:
    """One synthetic problem: matrix, GLE, context options and the algorithmic work of
    each kernel class per launch (for the roofline)."""

    def __init__(self, name, precision):
        self.name = name
        from paper_1402_2095_gb300 import fit
        self.M32 = self.M64 = self.csr = None
        self.nnz = 0
        if name == "dense4096":
            self.n, self.R, self.block = 4096, 256, 1000
            self.seed = syn.BASE_SEED + 1
            M, lam, _ = syn.dense_spd(self.n, 1.0, 1000.0, seed=self.seed)
            self.mu = float(np.median(lam))
            self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("fermi_b5_dense4096")
            # the fit is centred on this workload's own median eigenvalue
            if abs(self.fit["params"][1] - self.mu) > 1e-9 * self.mu:
                raise ValueError("stored Fermi fit is not centred on the median eigenvalue")
            self.M32 = M.astype(np.float32)
            self.precision = precision
            self.track, self.pairs = "all", None
            self.label = ("dense SPD N=4096, lambda log-uniform [1,1e3], Fermi beta=5 mu=median, "
                          "R=256, all elements")
            self.default_steps, self.cpu_replicas = 20000, 16
        elif name == "small_fp64":
            self.n, self.R, self.block = 32, 16, 1000
            self.seed = syn.BASE_SEED + 0
            M, lam, _ = syn.dense_spd(self.n, 1.0, 100.0, seed=self.seed)
            self.mu = None
            self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("inv_sqrt_1_100")
            self.M64 = M
            self.precision = "fp64"
            self.track, self.pairs = "all", None
            self.label = ("dense SPD N=32 FP64, lambda log-uniform [1,100], f=x^-1/2, R=16, "
                          "all 528 elements")
            self.default_steps, self.cpu_replicas = 100000, 16
        elif name == "lattice64":
            L = 64
            self.n, self.R, self.block = L ** 3, 64, 1000
            self.seed = syn.BASE_SEED + 2
            rowptr, col, val = syn.lattice_csr(L, seed=self.seed)
            self.csr = (rowptr, col, val.astype(np.float32), self.n)
            self.nnz = len(col)
            self.mu = 7.0
            self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("fermi_b2_lattice")
            self.precision = "fp32"
            self.track = "list"
            self.pairs = np.concatenate([syn.diag_pairs(self.n), syn.lattice_nn_pairs(L)])
            self.label = ("64^3 periodic lattice CSR (N=262144, 7-point), Fermi beta=2 mu=7, "
                          "R=64, diagonal + nearest-neighbour elements")
            self.default_steps, self.cpu_replicas = 2000, 4
        elif name == "m1":
            # the paper's logarithm benchmark: Tr ln M1 (Appendix M1: n^3 lattice, on-site
            # 100, hopping U[0,2] to six neighbour shells), ln fitted on [e, 100e], M1
            # scaled into it: Tr ln M1 = Tr ln(r M1) - N ln r
            import scipy.sparse as sp
            import scipy.sparse.linalg as spla
            n1 = 16
            self.n, self.R, self.block = n1 ** 3, 64, 1000
            self.seed = syn.BASE_SEED + 5
            rowptr, col, val = syn.m1_csr(n1, seed=self.seed)
            A = sp.csr_matrix((val, col, rowptr), shape=(self.n, self.n))
            lo = float(spla.eigsh(A, k=1, which="SA", return_eigenvectors=False, tol=1e-8)[0])
            hi = float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False, tol=1e-8)[0])
            self.spectrum = (lo, hi)
            self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("log_e_100e")
            self.r = float(np.e) * 1.0005 / lo             # r lo just above e
            if self.r * hi > 100 * np.e:
                raise ValueError("M1 spectrum wider than the fitted range")
            self.csr = (rowptr, col, (self.r * val).astype(np.float32), self.n)
            self.nnz = len(col)
            self.mu = None
            self.precision = "fp32"
            self.track, self.pairs = "diag", syn.diag_pairs(self.n)
            self.trace = ("log", self.r)
            self.label = (f"Tr ln M1, M1 = paper's Appendix lattice n={n1} (N={self.n}, 80 "
                          f"neighbours), ln fitted on [e,100e], r={self.r:.5f}, R=64, diagonal")
            self.default_steps, self.cpu_replicas = 20000, 4
        elif name == "m2":
            # the paper's exponential benchmark: Tr exp(-M2/100) (Appendix M2, eigenvalues
            # in (-300, 300)); exp(-x/100) fitted on [1, 601] for M2 + 301 I
            m = 2048
            self.n, self.R, self.block = m, 256, 1000
            self.seed = syn.BASE_SEED + 6
            M2 = syn.m2_dense(m, seed=self.seed)
            self.shift = 301.0
            self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("exp_001_1_601")
            self.M32 = (M2 + self.shift * np.eye(m)).astype(np.float32)
            self.mu = None
            self.precision = precision
            self.track, self.pairs = "diag", syn.diag_pairs(m)
            self.trace = ("exp", 0.01, self.shift)
            self.label = (f"Tr exp(-M2/100), M2 = paper's Appendix dense random (m={m}, "
                          f"eigenvalues in (-300,300)) + 301 I, exp(-x/100) fitted on [1,601], "
                          f"R=256, diagonal")
            self.default_steps, self.cpu_replicas = 20000, 8
        else:
            raise ValueError(name)
        if not hasattr(self, "trace"):
            self.trace = None

    def untransform(self, v):
        """The wanted trace from the sampled one (paper's inverse transforms)."""
        from paper_1402_2095_gb300 import transforms as tr
        if self.trace is None:
            return v
        if self.trace[0] == "log":
            return tr.log_trace_from_scaled(v, self.n, self.trace[1])
        return float(tr.exp_from_shifted(v, self.trace[1], self.trace[2]))

    def untransform_err(self, e):
        if self.trace is None or self.trace[0] == "log":
            return e
        return float(e * np.exp(self.trace[1] * self.trace[2]))

    def matrix_kwargs(self, device, pinned=False):
        import torch
        if self.csr is not None:
            return {"csr": self.csr}
        if self.precision == "fp64":
            return {"M": self.M64}
        t = torch.from_numpy(self.M32)
        if device:
            return {"M": t.cuda()}
        return {"M": t.pin_memory() if pinned else t}

    def element_pairs(self):
        if self.pairs is not None:
            return self.pairs
        return syn.upper_pairs(self.n)

    def oracle_matrix(self):
        if self.csr is not None:
            rowptr, col, val, n = self.csr
            return {"csr": (rowptr, col, val.astype(np.float64), n)}
        M = self.M64 if self.precision == "fp64" else self.M32.astype(np.float64)
        return {"M": M}

    def work(self, cls, info):
        """(bound, algorithmic amount per launch) of a kernel class."""
        n, R = self.n, self.R
        if cls in ("force_tc", "force_fp32"):
            return ("tensor" if cls == "force_tc" else "alu", 2.0 * n * n * R)
        if cls in ("syrk_tc", "syrk_fp32"):
            return ("tensor" if cls == "syrk_tc" else "alu", float(n) * (n + 1) * info["stack_cols"])
        if cls == "gle_dense":
            tc = self.precision in ("tf32", "bf16x3")
            op = 4 if tc else 0                                  # q^T operand of the force
            sample = 2 if tc and self.track == "all" else 4      # BF16 or FP32 stack
            zero = 4 if self.precision == "tf32" else 0          # zeros over MQ (reduce-add force)
            return ("hbm", float(28 + 24 + sample + op + zero) * n * R)
        if cls == "csr_step":
            return ("hbm", float(24 + 24 + 4) * n * R + 8.0 * self.nnz + 4.0 * n)
        if cls == "pair_accum":
            return ("hbm", 2.0 * 4 * info["stack_cols"] * len(self.element_pairs()))
        if cls == "fp64_dense":
            ns = 5
            per = 2.0 * n * n + 2 * 2 * (ns * ns + ns * (ns + 1) / 2) * n + 2.0 * n * (n + 1) / 2
            return ("fp64", info["steps_per_launch"] * R * per)
        return ("hbm", float("nan"))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


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
        # nvidia-smi's first query initialises NVML; let that finish before timing starts
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 10.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

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
def _traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu capture of this kernel on this
    workload ("name:precision"), or None when there is none or the kernel's source has
    changed since the capture (hash mismatch)."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) == 5 and f[0] == kernel and f[1] == workload:
            try:
                src = open(os.path.join(ROOT, f[2]), "rb").read()
            except OSError:
                return None
            if hashlib.sha256(src).hexdigest()[:16] == f[3]:
                return int(f[4])
    return None


def roofline(prof, wl, info, peaks, peak_kind):
    """Dominant kernel (largest total device time) against its bound."""
    name, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_s = ms / cnt / 1e3
    bound, amount = wl.work(name, info)
    tf32_ratio = 1.1 / 2.25           # nominal dense TF32 / BF16 tensor rate
    # the per-kernel times come from a pass of ~2000 steps (well under a second of tensor
    # work per kernel class), so the burst figure is the peak to compare with
    burst = peaks["bf16_tflops"]
    fp32_alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if bound == "tensor":
        # the accumulation pass multiplies BF16 samples; the force runs in the line's form
        tf = wl.precision == "tf32" and name != "syrk_tc"
        peak = burst * (tf32_ratio if tf else 1.0)
        out = {"bound": "tensor", "unit": "TFLOP/s", "achieved": amount / per_launch_s / 1e12,
               "peak": peak, "peak_source": f"{peak_kind} bf16 burst"
                                            + (" x 1.1/2.25 (TF32)" if tf else "")}
    elif bound == "alu":
        out = {"bound": "alu", "unit": "TFLOP/s", "achieved": amount / per_launch_s / 1e12,
               "peak": fp32_alu, "peak_source": "FP32 FMA: 152 SM x 128 lanes x 2 x max SM clock"}
    elif bound == "fp64":
        out = {"bound": "alu", "unit": "TFLOP/s", "achieved": amount / per_launch_s / 1e12,
               "peak": 1.25, "peak_source": "nominal FP64 1.25 TFLOP/s"}
    else:
        out = {"bound": "hbm", "unit": "GB/s", "achieved": amount / per_launch_s / 1e9,
               "peak": peaks["hbm_gbs"], "peak_source": f"{peak_kind} copy"}
    out["frac"] = out["achieved"] / out["peak"]
    out["kernel"] = name
    out["launch_us"] = per_launch_s * 1e6
    out["traffic"] = _traffic(name, f"{wl.name}:{wl.precision}")
    total = sum(x[0] for x in prof.values())
    out["share"] = {k: round(v[0] / total, 4) for k, v in prof.items()}
    return out


# ---------------------------------------------------------------------- CPU oracle
def _oracle(wl):
    from oracle.fth import OracleFTH
    R = min(wl.cpu_replicas, wl.R)
    return OracleFTH(**wl.oracle_matrix(), a_p=wl.a_p, c_p=wl.c_p, dt=wl.dt, replicas=R,
                     seed=wl.seed, block=wl.block, pairs=wl.element_pairs()), R


def cpu_baseline(wl, budget_s=CPU_BUDGET_S):
    """The FP64 oracle as it stands on the host cores, on the same matrix and GLE with
    a replica sample and the same tracked elements; timed for about budget_s."""
    o, R = _oracle(wl)
    o.run(1)
    steps, chunk, t0 = 0, 1, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.run(chunk)
        steps += chunk
        if time.perf_counter() - t0 < 0.1 * budget_s:
            chunk = min(chunk * 2, 4096)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": R * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{wl.name}: {R} of {wl.R} replicas, {len(wl.element_pairs())} elements, "
                      f"{steps} steps in {el:.1f} s"}


def _exact_values(wl, pairs, burnin, nacc, nsample=16, degree=400):
    """The oracle's exact values at the tracked elements: g (stationary), the expected
    running mean after `burnin` discarded and `nacc` accumulated samples from the zero
    state, and f (the wanted function); dense and small lattices by the FP64
    eigendecomposition (all elements), lattices too large for it by the Chebyshev route on
    a seeded sample of the elements (half diagonal, half off-diagonal).  Returns
    (index of the elements used, G, GM, F, info, eigenvalues or None)."""
    from oracle import gle, matfun
    t0 = time.perf_counter()
    T, S = gle.propagator(wl.a_p, wl.c_p, wl.dt)
    fk, fp = wl.fit["kind"], tuple(wl.fit.get("params", ()))
    if wl.csr is not None and wl.n > 8192:
        rng = np.random.default_rng(wl.seed)
        diag = np.flatnonzero(pairs[:, 0] == pairs[:, 1])
        off = np.flatnonzero(pairs[:, 0] != pairs[:, 1])
        h = nsample // 2
        pick = np.concatenate([rng.choice(diag, min(h, len(diag)), replace=False),
                               rng.choice(off, min(nsample - h, len(off)), replace=False)])
        rowptr, col, val, n_ = wl.oracle_matrix()["csr"]
        fns = [lambda x: gle.mode_response(x, T, S, wl.dt),
               lambda x: gle.mode_response_mean(x, T, S, wl.dt, burnin, nacc),
               lambda x: matfun.f_scalar(fk, x, fp)]
        (G, GM, F), tails = matfun.fn_elements_sparse(rowptr, col, val, n_, fns, pairs[pick],
                                                      degree=degree)
        info = {"sample": f"{len(pick)} of {len(pairs)} tracked elements, Chebyshev degree "
                          f"{degree} on the Gershgorin interval", "chebyshev_tail": max(tails),
                "oracle_s": time.perf_counter() - t0}
        return pick, G, GM, F, info, None
    om = wl.oracle_matrix()
    if "M" in om:
        M = om["M"]
    else:
        import scipy.sparse as sp
        rowptr, col, val, n_ = om["csr"]
        M = sp.csr_matrix((val, col, rowptr), shape=(n_, n_)).toarray()
    lam, U = np.linalg.eigh(M)
    t_eigh = time.perf_counter() - t0
    g = gle.mode_response(lam, T, S, wl.dt)
    gm = gle.mode_response_mean(lam, T, S, wl.dt, burnin, nacc)
    f = matfun.f_scalar(fk, lam, fp)
    ii, jj = pairs[:, 0], pairs[:, 1]
    n = M.shape[0]

    def elems(d):
        # U diag(d) U^T at the pairs: whole matrix when most elements are tracked,
        # else row pairs in chunks of ~64 MB
        if len(ii) * 8 > n * n:
            return ((U * d[None, :]) @ U.T)[ii, jj]
        out = np.empty(len(ii))
        ch = max(1, (1 << 23) // n)
        for c0 in range(0, len(ii), ch):
            a, b = ii[c0:c0 + ch], jj[c0:c0 + ch]
            out[c0:c0 + len(a)] = np.einsum("kj,kj->k", U[a] * d[None, :], U[b])
        return out

    info = {"sample": f"all {len(pairs)} tracked elements, FP64 eigendecomposition",
            "eigh_s": t_eigh, "oracle_s": time.perf_counter() - t0}
    return np.arange(len(pairs)), elems(g), elems(gm), elems(f), info, (lam, g, gm, f)


def exact_target(wl, pairs, acc):
    """Part of the CPU baseline: the oracle's exact values (see _exact_values) and each
    accuracy-pass estimate's error against them.  Per estimate: rel_err = ||est - E[est]||
    / ||g|| (E[est] the exact expected running mean after the pass's burn-in and
    accumulated samples), sigma_rel = ||errbar|| / ||g||, z2 = <((est - E[est]) / errbar)^2>
    (near 1 when the block error bars are right), steps_to_1e-3 = burn-in + accumulated x
    (sigma_rel / 1e-3)^2 (the statistical error falls as steps^-1/2 once the blocks are
    longer than the correlation time), time_to_1e-3 = that x the form's measured step
    time.  transient = ||E[est] - g|| / ||g|| (what the burn-in left), fit_bias = ||g - f||
    / ||f|| (the fitted GLE against the wanted function: against f itself 1e-3 is out of
    reach whenever this exceeds it)."""
    pick, G, GM, F, info, modes = _exact_values(wl, pairs, acc["burnin"], acc["accumulated"])
    ng = float(np.linalg.norm(G))
    out = dict(info)
    out.update({"burnin": acc["burnin"], "block": acc["block"], "accumulated": acc["accumulated"],
                "tau_max": acc["tau_max"],
                "transient": float(np.linalg.norm(GM - G)) / ng,
                "fit_bias": float(np.linalg.norm(G - F) / np.linalg.norm(F))})
    main = acc["runs"][acc["form"]]
    v, e = main["vals"][pick], main["errs"][pick]
    z = (v - GM) / e
    sig = float(np.linalg.norm(e)) / ng
    steps_to = acc["burnin"] + acc["accumulated"] * (sig / 1e-3) ** 2
    out[acc["form"]] = {
        "rel_err": float(np.linalg.norm(v - GM)) / ng, "sigma_rel": sig,
        "z2": float(np.mean(z * z)), "frac_abs_z_below_4": float(np.mean(np.abs(z) < 4.0)),
        "ms_per_step": main["ms_per_step"], "steps_to_1e-3": steps_to,
        "time_to_1e-3_s": steps_to * main["ms_per_step"] / 1e3}
    d = pairs[pick, 0] == pairs[pick, 1]
    if d.any() and not d.all():
        sd = float(np.linalg.norm(e[d]) / np.linalg.norm(G[d]))
        td = acc["burnin"] + acc["accumulated"] * (sd / 1e-3) ** 2
        out[acc["form"]].update({"sigma_rel_diag": sd, "steps_to_1e-3_diag": td,
                                 "time_to_1e-3_diag_s": td * main["ms_per_step"] / 1e3})
    for form, run in acc["runs"].items():
        if form == acc["form"]:
            continue
        # same seed, so the same noise: the difference of the two estimates after the same
        # samples is the precision difference of the two forms, not statistics
        diff = float(np.linalg.norm(run["vals"][pick] - acc["snapshot"][pick])) / ng
        out[form] = {
            "ms_per_step": run["ms_per_step"], "paired_steps": run["steps"],
            "paired_rel_diff_vs_" + acc["form"]: diff,
            "steps_to_1e-3": steps_to, "time_to_1e-3_s": steps_to * run["ms_per_step"] / 1e3,
            "note": "same dynamics and noise as the " + acc["form"] + " run, so the same error "
                    "bar per step; its time is that step count at this form's step time"}
    if acc.get("trace") is not None and modes is not None:
        lam, g, gm, f = modes
        tv, te = acc["trace"]
        tr_g, tr_gm, tr_f = float(np.sum(g)), float(np.sum(gm)), float(np.sum(f))
        sig_t = te / abs(tr_g)
        t_t = acc["burnin"] + acc["accumulated"] * (sig_t / 1e-3) ** 2
        out["trace"] = {
            "sampled": tv, "errbar": te, "exact_expected": tr_gm, "exact_g": tr_g,
            "exact_f": tr_f, "rel_err": abs(tv - tr_gm) / abs(tr_g), "sigma_rel": sig_t,
            "z": (tv - tr_gm) / te, "wanted": wl.untransform(tv),
            "wanted_exact": wl.untransform(tr_f), "steps_to_1e-3": t_t,
            "time_to_1e-3_s": t_t * main["ms_per_step"] / 1e3}
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "serving":
        print(json.dumps({"impl": "reference", "unavailable":
                          "serving stream: the FP64 oracle would need hours of host time to "
                          "serve the request stream once; per-step oracle baselines are the "
                          "dense4096, lattice64, small_fp64 and ragged512 reference lines"}),
              flush=True)
        return 0
    if args.workload == "ragged512":
        wl = Ragged()
        cb = cpu_baseline_ragged(wl, budget_s=REF_BUDGET_S, steps=args.steps)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": wl.count * wl.R / cb["value"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl.label}, "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    wl = Workload(args.workload, args.precision)
    o, R = _oracle(wl)
    o.run(min(max(args.warmup, 1), 2))
    # each step is a bounded sample (R of the workload's replicas, the same elements);
    # the run stops after REF_BUDGET_S if K steps would take longer
    steps, t0 = 0, time.perf_counter()
    while steps < args.steps and time.perf_counter() - t0 < REF_BUDGET_S:
        o.run(1)
        steps += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = R * steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": el / max(steps, 1) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.label, "n": wl.n, "replicas_sampled": R},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{wl.name}: {R} of {wl.R} replicas per step, "
                                   f"{len(wl.element_pairs())} elements, {steps} steps in "
                                   f"{el:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- ragged batches
class Ragged:
    """512 dense SPD problems, N_k = 64 u with u uniform on {1..16}, lambda log-uniform
    in [1, 1e2], Haar Q, f = x^-1/2 (one fitted GLE, s = 4), R = 32 replicas each,
    BF16x3 force, FP32 state; tracked: the diagonal plus 32 seeded off-diagonal pairs
    per problem; all problems stepped together by one problem pool (persistent force
    kernel over (problem, 128-row block) items, chunks of steps replayed from a captured
    CUDA graph, force configuration picked by the pool's autotuner)."""

    name = "ragged512"
    count, R, block, graph_steps = 512, 32, 1000, 50

    def __init__(self):
        from paper_1402_2095_gb300 import fit
        self.seed = syn.BASE_SEED + 3
        self.sizes = syn.ragged_sizes(self.count, seed=self.seed)
        self.a_p, self.c_p, self.dt, self.fit = fit.load_gle("inv_sqrt_1_100")
        self.block = calibrated_blocks(self.a_p, self.c_p, self.dt, self.fit["lam"])[2]
        self.mats, self.pairs = [], []
        for k, n in enumerate(self.sizes):
            M, _, _ = syn.dense_spd(int(n), 1.0, 100.0, seed=self.seed * 1000 + k)
            self.mats.append(M.astype(np.float32))
            self.pairs.append(np.concatenate([syn.diag_pairs(int(n)),
                                              syn.random_pairs(int(n), 32, seed=k)]))
        self.label = ("512 dense SPD, N = 64u (u uniform 1..16), lambda log-uniform [1,1e2], "
                      "f=x^-1/2, R=32 each, BF16x3 force, diagonal + 32 pairs each")
        self.default_steps = 4000

    def problem(self, k, seed_shift=0):
        return dict(M=self.mats[k], a_p=self.a_p, c_p=self.c_p, dt=self.dt,
                    seed=self.seed * 1000 + k + seed_shift, block=self.block,
                    pairs=self.pairs[k])

    def work(self, cls):
        """Algorithmic bytes per launch of each pool kernel class (all HBM-bound):
        force: the N(N+1)/2 distinct elements of the symmetric M as BF16 hi+lo (4 B each),
        q^T operand hi+lo in, M q out;
        gle: 60 B per (i, r) (q, p, s1..s4, M q in; q, p, s1..s4, sample, operand out);
        accumulate: the sample rows of every tracked pair."""
        N = self.sizes.astype(np.float64)
        R = self.R
        if cls == "pool_force":
            return float(np.sum(2.0 * N * (N + 1) + 4.0 * N * R + 4.0 * N * R))
        if cls == "pool_gle":
            return float(np.sum(60.0 * N * R))
        if cls == "pool_accum":
            return float(sum(2 * 4 * R * len(p) for p in self.pairs))
        return float("nan")


def run_ragged(args, rank, world, local):
    import torch
    from paper_1402_2095_gb300 import Pool
    wl = Ragged()
    steps = args.steps if args.steps is not None else wl.default_steps
    ws = 3 << 30
    pool = Pool(ws, replicas=wl.R, precision="bf16x3", max_problems=wl.count,
                graph_steps=wl.graph_steps)
    for k in range(wl.count):
        pool.add(**wl.problem(k), replica_offset=rank * wl.R)
    pool.run(args.warmup)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(pool.stream)
    pool.run(steps)
    ev1.record(pool.stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = pool.stats()
    prof = pool.profile(min(steps, 200))
    peaks, peak_kind = _peaks()
    name, (pms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_s = pms / cnt / 1e3
    achieved = wl.work(name) / per_launch_s / 1e9
    total = sum(v[0] for v in prof.values())
    roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peaks["hbm_gbs"],
            "peak_source": f"{peak_kind} copy", "frac": achieved / peaks["hbm_gbs"],
            "kernel": name, "launch_us": per_launch_s * 1e6, "traffic": _traffic(name, "ragged512:bf16x3"),
            "share": {k: round(v[0] / total, 4) for k, v in prof.items()}}
    pool.close()
    del pool
    torch.cuda.synchronize()

    # end to end through the public API: host matrices (pinned) in, every problem's elements out
    pinned = [torch.from_numpy(m).pin_memory() for m in wl.mats]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = Pool(ws, replicas=wl.R, precision="bf16x3", max_problems=wl.count,
             graph_steps=wl.graph_steps)
    hs = [g.add(**dict(wl.problem(k, seed_shift=1), M=pinned[k]), replica_offset=rank * wl.R)
          for k in range(wl.count)]
    e2e_steps = max(steps, E2E_MIN_STEPS)
    g.run(e2e_steps)
    read = {}
    for k, h in enumerate(hs):
        read[k] = g.elements(h, wl.pairs[k])
    t_e2e = time.perf_counter() - t0
    g.close()
    del pinned
    h2d = sum(m.nbytes for m in wl.mats) + sum(p.nbytes for p in wl.pairs)
    d2h = sum(len(p) * 3 * 8 for p in wl.pairs)

    value = wl.count * wl.R * steps * world / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": {"workload": wl.label, "problems": wl.count, "sum_n": int(wl.sizes.sum()),
                   "sum_n2": int(np.sum(wl.sizes.astype(np.int64) ** 2)),
                   "replicas_per_problem": wl.R, "precision": "bf16x3",
                   "graph_steps": wl.graph_steps, "tuned_variant": st["tuned_variant"],
                   "tuned_grid": st["tuned_grid"], "tuned_force_us": st["tuned_us"],
                   "gle_variant": st["gle_variant"], "tuned_gle_us": st["gle_us"],
                   "parallelism": f"replicas x{world}",
                   "l2": "per-step working set (M hi+lo upper blocks %.0f MB + state %.0f MB) > L2; "
                         "steps back to back" % (wl.work("pool_force") / 1e6,
                                                 wl.work("pool_gle") / 1e6)},
        "gpu_launches": 3 * steps,
        "clocks": clk,
        "roofline": roof,
        "e2e": {"value": wl.count * wl.R * e2e_steps * world / t_e2e, "unit": UNIT,
                "steps": e2e_steps, "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps},
    }
    if rank == 0 and world == 1 and not args.no_accuracy:
        # fixed-length pass with calibrated burn-in and blocks (independent of --steps)
        tau, burnin, block = calibrated_blocks(wl.a_p, wl.c_p, wl.dt, wl.fit["lam"])
        nblocks = args.accuracy_blocks
        pa = Pool(ws, replicas=wl.R, precision="bf16x3", max_problems=wl.count,
                  graph_steps=wl.graph_steps)
        hs = [pa.add(**dict(wl.problem(k, seed_shift=2), burnin=burnin, block=block))
              for k in range(wl.count)]
        nsteps = 1 + burnin + nblocks * block          # the first pool step is the prologue
        pa.run(nsteps)
        acc_read = {k: pa.elements(hs[k], wl.pairs[k]) for k in range(wl.count)}
        pa.close()
        line["accuracy"] = {"form": "bf16x3", "tau_max": tau, "burnin": burnin, "block": block,
                            "blocks": nblocks, "accumulated": nblocks * block, "steps": nsteps}
        if not args.no_cpu_baseline:
            line["accuracy"]["exact"] = exact_target_ragged(wl, acc_read, burnin,
                                                            nblocks * block, ms / steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_ragged(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def exact_target_ragged(wl, read, burnin, nacc, ms_per_step, nsample=8):
    """exact_target for the pool: on a seeded sample of problems, each problem's exact
    values by the oracle's eigendecomposition (g, the expected running mean after `burnin`
    discarded and `nacc` accumulated samples, f) at its tracked pairs, against the values
    and error bars the pool returned (`read[k]` = (values, errbars) of problem k).  Norms
    over the sample's elements together; all problems advance one step per pool step, so
    the time to 1e-3 is in pool steps: burn-in + nacc (sigma_rel / 1e-3)^2."""
    steps = nacc
    from oracle import gle, matfun
    t0 = time.perf_counter()
    pick = np.random.default_rng(wl.seed + 1).choice(wl.count, size=nsample, replace=False)
    T, S = gle.propagator(wl.a_p, wl.c_p, wl.dt)
    fk, fp = wl.fit["kind"], tuple(wl.fit.get("params", ()))
    G, GM, F, V, E, D = [], [], [], [], [], []
    for k in pick:
        k = int(k)
        lam, U = np.linalg.eigh(wl.mats[k].astype(np.float64))
        pr = wl.pairs[k]
        a, b = U[pr[:, 0]], U[pr[:, 1]]
        for out, d in ((G, gle.mode_response(lam, T, S, wl.dt)),
                       (GM, gle.mode_response_mean(lam, T, S, wl.dt, burnin, nacc)),
                       (F, matfun.f_scalar(fk, lam, fp))):
            out.append(np.einsum("kj,kj->k", a * d[None, :], b))
        V.append(read[k][0])
        E.append(read[k][1])
        D.append(pr[:, 0] == pr[:, 1])
    G, GM, F, V, E, D = (np.concatenate(x) for x in (G, GM, F, V, E, D))
    ng = float(np.linalg.norm(G))
    sig = float(np.linalg.norm(E)) / ng
    sig_d = float(np.linalg.norm(E[D]) / np.linalg.norm(G[D]))
    t_all = burnin + steps * (sig / 1e-3) ** 2
    t_d = burnin + steps * (sig_d / 1e-3) ** 2
    z = (V - GM) / E
    return {
        "sample": f"{nsample} of {wl.count} problems (seeded), {len(G)} tracked elements",
        "eigh_s": time.perf_counter() - t0, "burnin": burnin, "accumulated": nacc,
        "rel_err": float(np.linalg.norm(V - GM)) / ng, "sigma_rel": sig,
        "z2": float(np.mean(z * z)),
        "transient": float(np.linalg.norm(GM - G)) / ng,
        "fit_bias": float(np.linalg.norm(G - F) / np.linalg.norm(F)),
        "time_to_1e-3_s": t_all * ms_per_step / 1e3, "steps_to_1e-3": t_all,
        "sigma_rel_diag": sig_d, "steps_to_1e-3_diag": t_d,
        "time_to_1e-3_diag_s": t_d * ms_per_step / 1e3,
    }


def cpu_baseline_ragged(wl, budget_s=CPU_BUDGET_S, nsample=16, steps=None):
    """The oracle on a seeded random sample of the 512 problems (R = 32 each, the same
    tracked elements): replica-steps/s of the sample, an estimate for the whole mix."""
    from oracle.fth import OracleFTH
    pick = np.random.default_rng(wl.seed).choice(wl.count, size=nsample, replace=False)
    done, t_used = 0, 0.0
    per = budget_s / nsample
    for k in pick:
        kw = wl.problem(int(k))
        o = OracleFTH(M=kw["M"].astype(np.float64), a_p=wl.a_p, c_p=wl.c_p, dt=wl.dt,
                      replicas=wl.R, seed=kw["seed"], block=wl.block, pairs=kw["pairs"])
        o.run(1)
        n_steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < per and (steps is None or n_steps < steps):
            o.run(4)
            n_steps += 4
        t_used += time.perf_counter() - t0
        done += n_steps * wl.R
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{wl.name}: {nsample} of {wl.count} problems (seeded), R={wl.R} each, "
                      f"{done} replica-steps in {t_used:.1f} s"}


# ---------------------------------------------------------------------- serving
class Serving:
    """Poisson request stream at `rate` per second over an arrival window of `window`
    seconds.  Each request: 50 % dense SPD (N uniform in [128, 4096], lambda log-uniform
    in [1, 1e2], Haar Q), 50 % periodic lattice L^3 (L uniform in {16..48}, as the 64^3
    workload); f = x^-1/2 or Fermi beta = 2 (mu = median lambda = 10 dense, 7 lattice),
    50 / 50, each with the GLE fitted to its spectrum range; relative accuracy target t_hi
    or t_lo, 50 / 50;
    32 tracked elements (16 diagonal, 16 off-diagonal: random pairs dense, nearest
    neighbours lattice); R = 32 replicas; its own Philox key.  Matrices are drawn from
    a seeded set of `distinct` dense and lattice matrices generated before the run."""

    name = "serving"

    def __init__(self, rate=200.0, window=1.0, t_hi=0.1, t_lo=0.03, budget=40000, distinct=8):
        from paper_1402_2095_gb300 import fit
        self.seed = syn.BASE_SEED + 4
        g = np.random.default_rng(self.seed)
        self.rate, self.window, self.t_hi, self.t_lo, self.budget = rate, window, t_hi, t_lo, budget
        self.arrivals = syn.poisson_arrivals(rate, window, seed=self.seed)
        self.fits = {k: fit.load_gle(k) for k in ("inv_sqrt_1_100", "fermi_b2_1_100",
                                                   "inv_sqrt_lattice", "fermi_b2_lattice")}
        # blocks calibrated per fit (correlation time of p^2 over its range)
        self.blocks = {k: calibrated_blocks(a, c, dt, rep["lam"])[2]
                       for k, (a, c, dt, rep) in self.fits.items()}
        self.dense, self.lattice = [], []
        for k in range(distinct):
            n = int(g.integers(128, 4097))
            M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=self.seed * 100 + k)
            self.dense.append(M.astype(np.float32))
            L = int(g.integers(16, 49))
            rowptr, col, val = syn.lattice_csr(L, seed=self.seed * 100 + k)
            self.lattice.append((rowptr, col, val.astype(np.float32), L ** 3, L))
        self.reqs = []
        lattice_inv_sqrt = []
        for j in range(len(self.arrivals)):
            dense = bool(g.integers(0, 2))
            k = int(g.integers(0, distinct))
            fermi = bool(g.integers(0, 2))
            target = self.t_hi if g.integers(0, 2) else self.t_lo
            if dense:
                n = self.dense[k].shape[0]
                fname = "fermi_b2_1_100" if fermi else "inv_sqrt_1_100"
                pairs = np.concatenate([syn.diag_pairs(n)[g.choice(n, 16, replace=False)],
                                        syn.random_pairs(n, 16, seed=self.seed + j)])
                mat = {"M": self.dense[k]}
            else:
                rowptr, col, val, n, L = self.lattice[k]
                nn = syn.lattice_nn_pairs(L)
                pairs = np.concatenate([syn.diag_pairs(n)[g.choice(n, 16, replace=False)],
                                        nn[g.choice(len(nn), 16, replace=False)]])
                fname = "fermi_b2_lattice" if fermi else "inv_sqrt_lattice"
                mat = {"csr": (rowptr, col, val, n)}
                if not fermi:
                    lattice_inv_sqrt.append(j)
            a_p, c_p, dt, _ = self.fits[fname]
            self.reqs.append(dict(mat, a_p=a_p, c_p=c_p, dt=dt, seed=self.seed * 10000 + j,
                                  block=self.blocks[fname], pairs=pairs, target=target,
                                  max_steps=budget))
        self.lattice_inv_sqrt = lattice_inv_sqrt
        self.label = (f"Poisson {rate:g} req/s over {window:g} s ({len(self.reqs)} requests); 50% "
                      f"dense N~U[128,4096] / 50% lattice L~U{{16..48}}; f in {{x^-1/2, Fermi b=2}}; "
                      f"targets {t_hi:g}/{t_lo:g} (normwise rel. error bar over blocks of "
                      f"max(1000, 10 tau_max) samples), budget {budget} steps; 32 elements; "
                      f"R=32 each")


def run_serving(args, rank, world, local):
    import torch
    from paper_1402_2095_gb300 import Server
    wl = Serving(rate=args.rate, window=args.window, budget=args.budget)
    srv = Server(args.serve_gb << 30, replicas=32, precision="bf16x3", max_problems=1024,
                 graph_steps=0, chunk_steps=1000, min_blocks=4, max_bypass=8)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ids, nxt = [], 0
    c0 = srv.clock()
    steps_total, launches, peak_used, busy = 0, 0, 0, 0.0
    t_end_limit = c0 + args.serve_timeout
    while True:
        now = srv.clock() - c0
        while nxt < len(wl.reqs) and wl.arrivals[nxt] <= now:
            ids.append(srv.submit(**wl.reqs[nxt]))
            nxt += 1
        c = srv.step()
        if c["running"] or c["admitted"]:
            steps_total += 1000
            launches += 3 * 1000
        peak_used = max(peak_used, c["used_bytes"])
        if nxt == len(wl.reqs) and c["running"] == 0 and c["queued"] == 0:
            break
        if srv.clock() > t_end_limit:
            break
        if c["running"] == 0 and c["queued"] == 0 and nxt < len(wl.reqs):
            # idle until the next arrival
            time.sleep(max(0.0, min(0.01, wl.arrivals[nxt] - (srv.clock() - c0))))
    torch.cuda.synchronize()
    clk = clocks.stop()
    wall = srv.clock() - c0
    lat, states, rsteps, relerr, met = [], {}, [], [], []
    example = None
    served = {}
    for j, rid in enumerate(ids):
        info, v, e = srv.result(rid)
        if v is not None and info["state"] in ("done", "budget"):
            served[j] = (v, e, info["steps"])
        if v is not None and example is None and j in wl.lattice_inv_sqrt:
            # one returned element of a lattice x^-1/2 request
            example = {"request": j, "element": [int(x) for x in wl.reqs[j]["pairs"][0]],
                       "f_M": float(v[0]), "errbar": float(e[0])}
        states[info["state"]] = states.get(info["state"], 0) + 1
        if info["state"] in ("done", "budget"):
            lat.append(info["t_done"] - c0 - wl.arrivals[j])
            met.append(info["state"] == "done")
            rsteps.append(info["steps"])
            relerr.append(info["rel_err"])
    lat = np.asarray(lat)
    met = np.asarray(met, dtype=bool)

    def pct(x):
        return ({"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)),
                 "count": int(x.size)} if x.size else {"p50": None, "p99": None, "count": 0})

    replica_steps = 32 * float(np.sum(rsteps))
    srv.close()
    p50 = float(np.percentile(lat, 50)) if lat.size else None
    p99 = float(np.percentile(lat, 99)) if lat.size else None
    line = {
        "metric": "p99 request latency", "value": p99, "unit": "s", "n_gpus": world,
        "steps": steps_total, "warmup": 0, "ms_per_step": wall / max(steps_total, 1) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/f32",
        "data": "synthetic",
        "config": {"workload": wl.label, "requests": len(wl.reqs), "submitted": len(ids),
                   "blocks": wl.blocks,
                   "states": states, "chunk_steps": 1000, "min_blocks": 4,
                   "workspace_gb": args.serve_gb, "peak_used_gb": peak_used / 2 ** 30,
                   "l2": "resident working set of all admitted requests >> L2"},
        "latency_s": {"p50": p50, "p99": p99, "mean": float(lat.mean()) if lat.size else None,
                      "max": float(lat.max()) if lat.size else None,
                      "met_target": pct(lat[met]), "spent_budget": pct(lat[~met]),
                      "share_met": float(met.mean()) if met.size else None},
        "throughput": {"requests_per_s": len(lat) / wall, "replica_steps_per_s": replica_steps / wall,
                       "wall_s": wall},
        "retired_rel_err": {"median": float(np.median(relerr)) if relerr else None},
        "served_vs_exact": serving_exact(wl, served) if rank == 0 else None,
        "example_result": example,
        "gpu_launches": launches, "clocks": clk,
        "e2e": {"value": p99, "unit": "s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "latency is end to end: host matrices submitted through the public "
                        "API, results read back on retirement"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serving_exact(wl, served, nsample=6):
    """Served results against the oracle: on a seeded sample of the retired dense requests,
    each request's exact expected running mean after its own number of samples (FP64
    eigendecomposition, per-mode response of its GLE) at its tracked elements; the
    normwise relative error of the served values and their z-scores against it."""
    from oracle import gle
    dense = sorted(j for j in served if "M" in wl.reqs[j])
    if not dense:
        return None
    t0 = time.perf_counter()
    pick = np.random.default_rng(wl.seed + 2).choice(dense, size=min(nsample, len(dense)),
                                                     replace=False)
    z, num, den = [], 0.0, 0.0
    for j in pick:
        r = wl.reqs[int(j)]
        v, e, steps = served[int(j)]
        lam, U = np.linalg.eigh(np.asarray(r["M"], dtype=np.float64))
        T, S = gle.propagator(r["a_p"], r["c_p"], r["dt"])
        # the first pool step of a request is its prologue: steps - 1 samples
        gm = gle.mode_response_mean(lam, T, S, r["dt"], 0, int(steps) - 1)
        pr = np.asarray(r["pairs"])
        want = np.einsum("kj,kj->k", U[pr[:, 0]] * gm[None, :], U[pr[:, 1]])
        num += float(np.sum((v - want) ** 2))
        den += float(np.sum(want ** 2))
        z.append((v - want) / e)
    z = np.abs(np.concatenate(z))
    return {"requests": int(len(pick)), "elements": int(z.size), "rel_err": (num / den) ** 0.5,
            "max_abs_z": float(np.max(z)), "frac_abs_z_below_4": float(np.mean(z < 4.0)),
            "eigh_s": time.perf_counter() - t0}


# ---------------------------------------------------------------------- accuracy pass
def calibrated_blocks(a_p, c_p, dt, lam_range):
    """(tau_max, burn-in, block) from the fitted GLE's integrated correlation time of the
    sampled p^2 over the spectral range, in samples (the library's exact per-mode
    response, fth_gle_response): burn-in 10 tau_max (the transient of the running mean
    falls as exp(-steps / tau)), blocks max(1000, 10 tau_max) samples (block means then
    nearly independent, so the block error bar is not optimistic)."""
    from paper_1402_2095_gb300 import binding
    lo, hi = lam_range
    lams = np.exp(np.linspace(np.log(lo), np.log(hi), 240))
    _, tau = binding.gle_response(a_p, c_p, dt, lams, tau=True)
    t = float(np.max(tau))
    return t, int(np.ceil(10 * t)), max(1000, int(np.ceil(10 * t)))


def accuracy_pass(wl, ctx_kw, stream, nblocks, compare):
    """Fixed-length runs for the time-to-1e-3 figures, independent of --steps and outside
    the timed region: the line's precision form from the zero state with the calibrated
    burn-in and `nblocks` calibrated blocks, its estimates read after one block (snapshot)
    and at the end; each form in `compare` on the same seed (same noise) for burn-in plus
    one block, timed, so the two estimates differ by precision alone."""
    import torch
    from paper_1402_2095_gb300 import FTH
    tau, burnin, block = calibrated_blocks(wl.a_p, wl.c_p, wl.dt, wl.fit["lam"])
    pairs = wl.element_pairs()
    kw = dict(ctx_kw, burnin=burnin, block=block, seed=wl.seed + 2)

    def timed(ctx, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # the step time of each form is taken over sampled steps only (after the burn-in, whose
    # steps skip the accumulation work), so it is the step time of a run that accumulates
    f = FTH(**wl.matrix_kwargs(device=True), **kw)
    fid = f.add_trace() if wl.trace is not None else None
    timed(f, burnin)
    ms_first = timed(f, block)
    snap = f.elements(pairs)[0]
    ms_rest = timed(f, (nblocks - 1) * block) if nblocks > 1 else 0.0
    vals, errs = f.elements(pairs)
    steps = burnin + nblocks * block
    f.poll()
    out = {"form": wl.precision, "tau_max": tau, "burnin": burnin, "block": block,
           "blocks": nblocks, "accumulated": nblocks * block, "snapshot": snap,
           "trace": f.functional(fid) if fid is not None else None,
           "runs": {wl.precision: {"vals": vals, "errs": errs, "steps": steps,
                                   "ms_per_step": (ms_first + ms_rest) / (nblocks * block)}}}
    f.close()
    del f
    for form in compare:
        g = FTH(**wl.matrix_kwargs(device=True), **dict(kw, precision=form))
        timed(g, burnin)
        ms2 = timed(g, block)
        v2, e2 = g.elements(pairs)
        g.poll()
        out["runs"][form] = {"vals": v2, "errs": e2, "steps": burnin + block,
                             "ms_per_step": ms2 / block}
        g.close()
        del g
    return out


def accuracy_summary(acc):
    """The JSON-safe part of an accuracy pass (no arrays)."""
    return {k: v for k, v in acc.items() if k not in ("snapshot", "runs", "trace")}


# ---------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense4096",
                    choices=["dense4096", "small_fp64", "lattice64", "ragged512", "serving", "m1",
                             "m2"])
    ap.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    ap.add_argument("--window", type=float, default=1.0, help="serving: arrival window (s)")
    ap.add_argument("--budget", type=int, default=40000, help="serving: step budget per request")
    ap.add_argument("--serve-gb", type=int, default=64, help="serving: pool workspace (GiB)")
    ap.add_argument("--serve-timeout", type=float, default=300.0, help="serving: wall limit (s)")
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the fixed-length accuracy pass (time to 1e-3)")
    ap.add_argument("--accuracy-blocks", type=int, default=12,
                    help="calibrated blocks in the accuracy pass")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 20000
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
    if args.workload in ("ragged512", "serving"):
        rc = (run_ragged if args.workload == "ragged512" else run_serving)(args, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return rc
    wl = Workload(args.workload, args.precision)
    # blocks as long as the calibrated accuracy pass uses (the flush cost per step is then
    # that of a real run); no burn-in, so every timed step accumulates its sample
    wl.tau, _, wl.block = calibrated_blocks(wl.a_p, wl.c_p, wl.dt, wl.fit["lam"])
    steps = args.steps if args.steps is not None else wl.default_steps
    stream = torch.cuda.current_stream()
    ctx_kw = dict(a_p=wl.a_p, c_p=wl.c_p, dt=wl.dt, replicas=wl.R, seed=wl.seed,
                  precision=wl.precision, track=wl.track, pairs=wl.pairs, block=wl.block,
                  stream=stream, replica_offset=rank * wl.R)
    f = FTH(**wl.matrix_kwargs(device=True), **ctx_kw)
    if wl.trace is not None:
        f.add_trace()
    f.run(args.warmup)
    torch.cuda.synchronize()
    l0 = f.info()["launches"]

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    f.run(steps)
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

    # per-kernel device time, CUDA events on each launching stream (separate pass)
    prof_steps = min(steps, 2000)
    f.profile(True)
    f.run(prof_steps)
    prof = f.profile_read()
    f.profile(False)
    peaks, peak_kind = _peaks()
    n64 = prof.get("fp64_dense", (0.0, 1))[1]
    # staged columns per accumulation pass (the library's default stack): 4096 BF16 columns
    # on the tensor-core paths, 2048 FP32 on the FFMA path, 4 samples for element lists
    tc_all = wl.track == "all" and wl.precision in ("tf32", "bf16x3")
    cols = 4096 if tc_all else 2048
    info = {"stack_cols": (cols // wl.R) * wl.R if wl.track == "all" else 4 * wl.R,
            "steps_per_launch": prof_steps / max(n64, 1)}
    roof = roofline(prof, wl, info, peaks, peak_kind)

    # end to end through the public API with host buffers: matrix in, results out
    pairs = wl.element_pairs()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = FTH(**wl.matrix_kwargs(device=False, pinned=True), **dict(ctx_kw, seed=wl.seed + 1))
    gfid = g.add_trace() if wl.trace is not None else None
    e2e_steps = max(steps, E2E_MIN_STEPS)
    g.run(e2e_steps)
    vals, errs = g.elements(pairs)
    trace_est = g.functional(gfid) if gfid is not None else None
    t_e2e = time.perf_counter() - t0
    if wl.csr is not None:
        h2d = wl.csr[0].nbytes + wl.csr[1].nbytes + wl.csr[2].nbytes + pairs.nbytes
    elif wl.precision == "fp64":
        h2d = wl.M64.nbytes
    else:
        h2d = wl.M32.nbytes
    h2d += pairs.shape[0] * 8                      # element indices of the results
    d2h = pairs.shape[0] * 3 * 8                   # (mean, M2, partial) per element
    g.close()
    del g

    value = wl.R * steps * world / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[wl.precision], "data": "synthetic",
        "config": {"workload": wl.label, "n": wl.n, "replicas_per_gpu": wl.R,
                   "precision": wl.precision, "track": wl.track, "s": 4, "dt": wl.dt,
                   "block": wl.block, "tau_max": wl.tau, "mu": wl.mu,
                   "fit": {k: wl.fit.get(k) for k in ("max_rel_err", "rms_rel_err", "max_abs_err",
                                                      "objective")},
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "e2e": {"value": wl.R * e2e_steps * world / t_e2e, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps},
    }
    if wl.name == "dense4096":
        sc = info["stack_cols"]
        line["config"]["l2"] = (
            "per-step working set > L2: M %d MB + state %d MB + staged samples %d MB + partial "
            "sums %d MB; steps back to back" % (
                wl.M32.nbytes >> 20, (8 * wl.n * wl.R * 4) >> 20,
                (wl.n * sc * (2 if tc_all else 4)) >> 20,
                ((wl.n // 128) * (wl.n // 128 + 1) // 2 * 128 * 128 * 4) >> 20))
    elif wl.name == "lattice64":
        line["config"]["l2"] = "state 805 MB per step > L2 (129 MB); steps back to back"
    elif wl.name in ("m1", "m2"):
        planes = (8 if wl.csr is not None else 9) * wl.n * wl.R * 4
        mbytes = 8 * wl.nnz if wl.csr is not None else wl.M32.nbytes
        line["config"]["l2"] = ("per-step working set %.0f MB (matrix %.0f MB + state) is below L2 "
                                "(129 MB): L2-resident by the workload's size, no flush between "
                                "steps" % ((planes + mbytes) / 1e6, mbytes / 1e6))
    else:
        line["config"]["l2"] = ("whole problem fits on chip (N=32): FP64 state in registers and "
                                "shared memory for the whole segment; no HBM traffic per step")
    if trace_est is not None:
        line["estimate"] = {"sampled_trace": trace_est[0], "sampled_errbar": trace_est[1],
                            "trace": wl.untransform(trace_est[0]),
                            "errbar": wl.untransform_err(trace_est[1]), "steps": e2e_steps}
    if rank == 0 and world == 1 and not args.no_accuracy:
        # time to 1e-3: a fixed-length pass of its own (calibrated burn-in and blocks),
        # the plain FP32 force beside the tensor-core forms
        compare = ["fp32"] if wl.precision in ("tf32", "bf16x3") else []
        acc = accuracy_pass(wl, ctx_kw, stream, args.accuracy_blocks, compare)
        line["accuracy"] = accuracy_summary(acc)
        if not args.no_cpu_baseline:
            line["accuracy"]["exact"] = exact_target(wl, pairs, acc)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
