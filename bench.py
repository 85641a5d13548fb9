"""Benchmark of the LAPS hot path on GB300: one JSON line on stdout.

A step is one complete LAPS run (Algorithm 1: initialisation, the unadjusted
phase, the switch, the adjusted phase, the samples) of the batched workload:
64 independent diagonal Gaussians of uneven dimension (d log-uniform in
[10, 2000], condition number log-uniform in [1e2, 1e4], 512..4096 chains) plus
one d = 10^4 Gaussian with 16384 chains, 234.6 M coordinates in all, every
problem 2000 integrator steps, all in one persistent launch per graph replay.
The paper's switch rule does not fire at these ensemble sizes (its window
statistic stays above 0.01), so the timed runs switch at the first full window
(step 400, the paper's "number of unadjusted steps" ablation knob) and run
MAMS proposals (MN2 for d <= 200, MN4 above) for the remaining steps.

value      chain-gradient-evals/s = sum over problems of M x gradient
           evaluations per chain / time of the whole run (laps_batch_init +
           laps_batch_run), initial positions resident on the device, CUDA
           events on the launching stream.  The state (1.9 GB) is larger than
           L2, so no flush is needed between runs.
e2e        the same metric through the batch entry points with host buffers:
           the initial positions copied in from pinned host memory, every
           problem's samples (laps_batch_sample) copied back, inside the timed
           region.
time_to_b2 per run, the device time from laps_batch_init until every problem's
           b^2_avg (Eq. "bias", against the closed-form moments) is below 0.01.
roofline   batch_kernel against the FP32 ALU issue rate: algorithmic operations
           of the run (the per-coordinate counts below) over the kernel's own
           duration (CUDA events around every launch of a whole run), against
           SMs x 128 lanes x the measured clock; beside it the counted
           instructions (ncu) and the algorithmic HBM bytes.
cpu_baseline  the FP64 oracle on the host cores on a bounded sample.

The register-resident form (banana d = 100, M = 4096, 5000 steps), the
logistic regression in its precisions, the ill-conditioned Gaussian and the
full-rank proxy are measured in the same run and reported under "forms".

--impl reference runs the oracle (the only reference this path has) instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import dataclasses
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chain-gradient-evals/sec and wall time to second-moment bias^2<0.01, 1 GB300"
UNIT = "chain-grad-evals/s"
BATCH = dict(name="batch64", n_steps=2000, switch_at=400, iters_per_launch=64)
RESIDENT = dict(name="banana_d100", d=100, M=4096, n_steps=5000, switch_at=1000)
# Algorithmic ALU operations per coordinate (one FP32 lane operation each):
# an O map is 48 (a quarter Philox4x32-10 call ~25 integer operations, half a
# Box-Muller pair ~17, uniforms 3, the O arithmetic 3), a B map 4, an A map
# with the target's gradient and log-p change 7 (banana and diagonal Gaussian
# alike), the ensemble sums 6 per step (y, y^2, g, y g) in the resident kernel
# and 2 (y, y^2) in the batch.
OPS_O, OPS_B, OPS_A = 48.0, 4.0, 7.0
ALU_OPS_LF = 2 * OPS_O + 2 * OPS_B + OPS_A + 6.0            # resident: 117 per step (1 gradient)
ALU_OPS_MN2_PER_GRAD = (2 * OPS_O + 3 * OPS_B + 2 * OPS_A) / 2  # 61
BATCH_OPS_LF = 2 * OPS_O + 2 * OPS_B + OPS_A + 2.0          # 113 per step (1 gradient)
BATCH_OPS_STEP = {1: 2 * OPS_O + 3 * OPS_B + 2 * OPS_A,     # MN2: 122 per step (2 gradients)
                  2: 2 * OPS_O + 6 * OPS_B + 5 * OPS_A}     # MN4: 155 per step (5 gradients)


def _rank_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def _max_over_ranks(x: float) -> float:
    """The largest value over the ranks of the process group (a job's time is
    its slowest rank's); x itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x: float) -> float:
    """The sum of x over the ranks of the process group; x itself without a
    group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8
                          for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


RESIDENT_SRC = ("laps_resident_kernel.cuh", "laps_resident.cuh", "laps_finalise.cuh", "laps_device.cuh",
                "laps_params.h")
BATCH_SRC = ("laps_batch.cu", "laps_resident.cuh", "laps_finalise.cuh", "laps_device.cuh", "laps_params.h")


def _kernel_source_hash(files=RESIDENT_SRC) -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_16696_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded(kernel: str, name: str = "resident_traffic.txt", files=RESIDENT_SRC):
    """The figures recorded for `kernel` in profiles/<name> from one ncu
    capture, or None when the kernel sources changed after that capture."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    cur = _kernel_source_hash(files)
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == cur:
            return [float(v) for v in f[2:]]
    return None


def _recorded_traffic(kernel: str):
    """DRAM bytes per launch of the resident kernel (profiles/resident_traffic.txt)."""
    r = _recorded(kernel)
    return r[0] if r else None


def _cpu_baseline(pr, seconds_hint=True, single_thread=False, grads_to_b2=None):
    """The oracle, as it stands, on the host cores: the first 500 unadjusted
    iterations of the same ensemble (all M chains).  single_thread adds the same
    on one core (first 50 iterations); grads_to_b2 (gradients per chain the GPU
    run needed to reach b^2 < 0.01) adds the oracle's projected time to it."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    tg = oracle.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb,
                             funnel_sv=pr.funnel_sv)

    def rate(n_it):
        run = oracle.OracleLAPS(tg, pr.x0, seed=0, n_total_steps=pr.n_steps)
        t0 = time.perf_counter()
        run.iterate(n_it)
        dt = time.perf_counter() - t0
        return pr.M * (run.trace[-1]["grads"] - 1) / dt, dt

    n_it = 500
    v, dt = rate(n_it)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "FP64 oracle, %d chains x first %d unadjusted iterations of %s (%.1f s)"
                     % (pr.M, n_it, pr.name, dt)}
    if grads_to_b2:
        out["projected_time_to_b2_s"] = pr.M * grads_to_b2 / v
    if single_thread:
        oracle.set_threads(1)
        v1, dt1 = rate(50)
        oracle.set_threads(cores)
        out["single_thread"] = {"value": v1, "cores": 1,
                                "sample": "first 50 unadjusted iterations (%.1f s)" % dt1}
        if grads_to_b2:
            out["single_thread"]["projected_time_to_b2_s"] = pr.M * grads_to_b2 / v1
    return out


def _oracle_rates():
    """The oracle, as it stands, on all host cores on a short slice of each of
    the other workloads (chain-gradient-evals/s; the slices are stated): the
    Gaussian (M = 256) and the funnel (M = 4096) for 50 and 20 unadjusted
    iterations, the logistic regression (M = 8192, n = 10^4) for 2, the batch's
    64 small problems for 1, and its d = 10^4 problem for 1 on 1024 of its chains."""
    import oracle
    from paper_2601_16696_gb300 import workloads
    cores = oracle.set_threads(os.cpu_count() or 1)

    def ot(pr):
        if pr.kind == workloads.LOGREG:
            return oracle.OracleTarget(pr.kind, pr.d, X=pr.X, y=pr.y, prior_var=pr.prior_var)
        return oracle.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb,
                                   funnel_sv=pr.funnel_sv)

    def rate(probs, n_it):
        evals, dt = 0, 0.0
        for k, pr in enumerate(probs):
            run = oracle.OracleLAPS(ot(pr), pr.x0, seed=0, pid=k, n_total_steps=pr.n_steps)
            t0 = time.perf_counter()
            run.iterate(n_it)
            dt += time.perf_counter() - t0
            evals += pr.M * (run.trace[-1]["grads"] - 1)
        return {"value": evals / dt, "unit": UNIT, "seconds": dt}

    out = {"cores": cores, "kind": "oracle"}
    out["gauss_d100_M256"] = rate([workloads.gauss_diag()], 50) | {"sample": "50 unadjusted iterations"}
    out["funnel_d101_M4096"] = rate([workloads.funnel()], 20) | {"sample": "20 unadjusted iterations"}
    out["logreg_d101_n10000_M8192"] = rate([workloads.logreg()], 2) | {"sample": "2 unadjusted iterations"}
    probs = workloads.batch64()
    out["batch64_small"] = rate(probs[:-1], 1) | {"sample": "1 unadjusted iteration of the 64 small problems"}
    big = dataclasses.replace(probs[-1], M=1024, x0=probs[-1].x0[:1024])
    out["batch64_big_d10000"] = rate([big], 1) | {"sample": "1 unadjusted iteration of its first 1024 chains"}
    return out


def _probe_peaks(stream):
    """Throughput probes of this GPU (laps_measure_peaks), and cuBLAS TF32 and
    FP64 GEMM throughput through torch (library GEMMs, for the tensor-core rates
    of those types; 8192^3 TF32, 4096^3 FP64)."""
    import torch
    from paper_2601_16696_gb300 import laps
    out = laps.measure_peaks(stream)

    def gemm_tflops(n, dtype, reps):
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        torch.matmul(a, b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        out["tf32_gemm_tflops"] = gemm_tflops(8192, torch.float32, 10)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["fp64_gemm_tflops"] = gemm_tflops(4096, torch.float64, 3)
    return out


def _batch_config(probs, extra=None):
    coords = sum(p.d * p.M for p in probs)
    cfg = {"workload": "batch64: 64 diagonal Gaussians, d log-uniform in [10, 2000], condition "
                       "1e2..1e4, M in {512..4096}, + d=10000 M=16384; %d steps each" % BATCH["n_steps"],
           "problems": len(probs), "coordinates": coords, "chains": sum(p.M for p in probs),
           "switch": "after %d unadjusted steps (the first full window; the paper's rule does not "
                     "fire at these ensemble sizes)" % BATCH["switch_at"],
           "l2": "not flushed: the state (%.1f GB) is larger than L2" % (8.0 * coords / 1e9)}
    cfg.update(extra or {})
    return cfg


def _batch_oracle(probs, total_chain_grads=None, iters=1):
    """The oracle, as it stands, on all host cores on a bounded sample of the
    batch: `iters` unadjusted iterations (one gradient per chain each) of each
    of the 64 small problems with all their chains, and of the d = 10^4 problem
    on its first 1024 chains.  total_chain_grads (the GPU run's) adds the
    oracle's projected time for a whole run."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    evals, dt = 0, 0.0
    for k, pr in enumerate(probs):
        if pr.d >= 10000:
            pr = dataclasses.replace(pr, M=1024, x0=pr.x0[:1024])
        tg = oracle.OracleTarget(pr.kind, pr.d, prec=pr.prec)
        run = oracle.OracleLAPS(tg, pr.x0, seed=0, pid=k, n_total_steps=pr.n_steps)
        t0 = time.perf_counter()
        run.iterate(iters)
        dt += time.perf_counter() - t0
        evals += pr.M * (run.trace[-1]["grads"] - 1)
    v = evals / dt
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
           "sample": "FP64 oracle, %d unadjusted iteration(s) of the 64 small problems (all chains) "
                     "and of the d = 10^4 problem on 1024 of its chains: %d chain-gradient "
                     "evaluations in %.2f s" % (iters, evals, dt)}
    if total_chain_grads:
        out["projected_run_s"] = total_chain_grads / v
    return out


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    from paper_2601_16696_gb300 import workloads
    probs = workloads.batch64(n_steps=BATCH["n_steps"])
    vals = [_batch_oracle(probs) for _ in range(args.warmup + args.steps)]
    timed = vals[args.warmup:]
    v = statistics.mean(r["value"] for r in timed)
    ms = statistics.mean(1e3 * r["seconds"] for r in timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": _batch_config(probs),
            "run": {"parallelism": "host cores (the oracle)"},
            "cpu_baseline": {k: timed[-1][k] for k in ("kind", "cores", "sample")} | {"value": v,
                                                                                    "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)


def _forms(flush, stream, mhz, seed0):
    """The other forms of the path, measured in the same run and reported
    beside the headline: the logistic regression (d = 101 with intercept,
    n = 10^4 rows, M = 8192) with the BF16 tensor-core contraction in the
    unadjusted phase beside the all-FP32 form; the rotated ill-conditioned
    Gaussian (d = 100, M = 4096, dense precision).
    Each: chain-gradient evaluations per second of a whole run, wall time to
    b^2 < 0.01, and the dominant kernel against its roofline.  Also the cost of
    an unadjusted iteration with the full-rank bias proxy (K = 20, 100)."""
    import torch
    from paper_2601_16696_gb300 import laps, workloads
    pk = _peaks()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = nsm * 128 * 2 * mhz * 1e6 / 1e12  # TFLOP/s, FMA lanes x 2 x clock

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed_ms(fn):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    out = {}
    # ---- logistic regression
    pr = workloads.logreg(with_truth=True)
    truth = "Laplace approximation of the posterior (FP64)"
    ref = workloads.logreg_reference_moments()
    if ref is not None:
        pr.Ex2, pr.Varx2 = ref
        truth = ("importance sampling from the Laplace Gaussian, FP64 "
                 "(tests/golden/logreg_d101_n10000_moments.txt)")
    tg = laps.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    n = pr.X.shape[0]
    flops = 4.0 * pr.M * n * pr.d  # Z = W X^T and G = R X per gradient of the ensemble
    lr = {"workload": "logreg_d%d_n%d_M%d_%dsteps" % (pr.d, n, pr.M, pr.n_steps),
          "b2": "b2_max", "truth": truth, "switch": "paper rule (max delta < 0.01)"}
    kernels = {0: "logreg_grad_f32_kernel<128>", 1: "logreg_grad_mma_kernel<128>",
               2: "logreg_grad_x3_kernel<128>"}
    for name, prec in (("mixed", 1), ("fp32", 0), ("bf16x3", 2)):
        for _ in range(3):
            tg.logp_grad(x0, precision=prec)
        reps = 10
        gms = timed_ms(lambda: [tg.logp_grad(x0, precision=prec) for _ in range(reps)]) / reps
        tg.check()
        # the whole 2000-step run (no early stop); the time to b^2_max < 0.01 is
        # the device time from laps_init to the first iteration below it
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, precision=prec, stop_b2_max=1)
        s.set_truth(pr.Ex2, pr.Varx2)
        s.init(x0, seed=seed0)
        s.step(3)  # warm-up of the launch sequence
        run_ms = timed_ms(lambda: (s.init(x0, seed=seed0 + 1), s.run()))
        st = s.stats()
        achieved = flops / (gms * 1e-3) / 1e12
        # the three-term form runs six BF16 products per FP32-accurate product
        peak = {0: fp32_peak, 1: pk["bf16_tflops"], 2: pk["bf16_tflops"] / 6.0}[prec]
        lr[name] = {
            "value": pr.M * st["grads"] / (run_ms * 1e-3), "unit": UNIT,
            "run_ms": run_ms, "grads_per_chain": st["grads"], "t": st["t"], "phase": st["phase"],
            "time_to_b2_ms": st["b2_first_ns"] / 1e6 if st["b2_first_t"] >= 0 else None,
            "grads_to_b2": st["b2_first_grads"] if st["b2_first_t"] >= 0 else None,
            "b2_max_final": st["b2_max"],
            "roofline": {"bound": "alu" if prec == 0 else "tensor", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "kernel": kernels[prec],
                         "timed": "laps_target_logp_grad_prec (points packed, contraction, "
                                  "partials summed), %.3f ms per call" % gms,
                         "peak_basis": {0: "%d SMs x 128 FP32 FMA lanes x 2 x %.0f MHz" % (nsm, mhz),
                                        1: "measured bf16 burst (MEASURED_PEAKS.json)",
                                        2: "measured bf16 burst / 6 (six BF16 products per "
                                           "FP32-accurate product)"}[prec]}}
    out["logreg"] = lr
    # ---- the logistic regression's adjusted phase: the switch forced after 100
    # unadjusted steps (the paper's rule does not fire on this workload), then
    # MAMS proposals to the end of the run; the adjusted phase's contraction on
    # the CUDA cores (mixed) or on the tensor cores at FP32 accuracy
    adj = {"workload": "logreg_d%d_n%d_M%d_%dsteps, switch forced at step 100" % (pr.d, n, pr.M, pr.n_steps)}
    for name, prec in (("mixed", 1), ("mixed_bf16x3", 3)):
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, precision=prec, force_switch_at=100)
        s.set_truth(pr.Ex2, pr.Varx2)
        s.init(x0, seed=seed0)
        s.step(3)
        run_ms = timed_ms(lambda: (s.init(x0, seed=seed0 + 1), s.run()))
        st = s.stats()
        tail = [r["acc"] for r in s.trace() if r["phase"] == 1 and not r["adapting"]]
        adj[name] = {"value": pr.M * st["grads"] / (run_ms * 1e-3), "unit": UNIT, "run_ms": run_ms,
                     "grads_per_chain": st["grads"], "t": st["t"], "phase": st["phase"],
                     "acceptance": float(statistics.mean(tail)) if tail else None,
                     "b2_max_final": st["b2_max"]}
    tg.check()
    out["logreg_adjusted"] = adj
    # ---- the rotated ill-conditioned Gaussian (dense precision, streamed path)
    pr = workloads.icg()
    tg = laps.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    for _ in range(3):
        tg.logp_grad(x0)
    reps = 20
    gms = timed_ms(lambda: [tg.logp_grad(x0) for _ in range(reps)]) / reps
    runs = {}
    for streamed in (1, 0):  # the streamed path, then the default (register-resident at d = 100)
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, stop_b2_max=1,  # b2_first on b^2_max
                         dense_streamed=streamed)
        s.set_truth(pr.Ex2, pr.Varx2)
        s.init(x0, seed=seed0)
        s.step(3)
        runs[streamed] = timed_ms(lambda: (s.init(x0, seed=seed0 + 1), s.run()))
    run_ms = runs[0]
    st = s.stats()
    flops = 2.0 * pr.M * pr.d * pr.d  # the contraction -P x of every chain, per gradient
    achieved = flops / (gms * 1e-3) / 1e12
    out["icg"] = {
        "workload": "icg_d%d_M%d_%dsteps (cond %.2g)" % (pr.d, pr.M, pr.n_steps, pr.extra["cond"]),
        "value": pr.M * st["grads"] / (run_ms * 1e-3), "unit": UNIT, "run_ms": run_ms,
        "path": "register-resident" if s.launch_info()["resident"] else "streamed",
        "run_ms_streamed_path": runs[1],
        "grads_per_chain": st["grads"], "t": st["t"], "phase": st["phase"],
        "time_to_b2_ms": st["b2_first_ns"] / 1e6 if st["b2_first_t"] >= 0 else None,
        "grads_to_b2": st["b2_first_grads"] if st["b2_first_t"] >= 0 else None, "b2": "b2_max",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "kernel": "gauss_dense_grad_kernel<4,2> (the streamed path's gradient)",
                     "timed": "laps_target_logp_grad (points packed, contraction, partials "
                              "unpacked), %.3f ms per call; 2 M d^2 algorithmic FLOP, the "
                              "compensated accumulation's extra operations not counted" % gms,
                     "peak_basis": "%d SMs x 128 FP32 FMA lanes x 2 x %.0f MHz" % (nsm, mhz)}}
    # ---- the full-rank bias proxy: unadjusted iterations on the headline ensemble
    pr = workloads.banana()
    tg = laps.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    fr = {"workload": "banana_d100_M4096, unadjusted iterations at a fixed step size"}
    for K in (0, 20, 100):
        s = laps.Sampler(tg, pr.M, n_total_steps=5000, fixed_eps=0.01, dtilde_K=K)
        s.init(x0, seed=seed0)
        s.step(20)
        fr["us_per_iteration_K%d" % K] = timed_ms(lambda: s.step(500)) / 500 * 1e3
    out["fullrank"] = fr
    return out


def ncu_case_form(which: str):
    """No timing: small cases of the other kernels, for ncu captures (a few hundred
    MB on the device at most).  logreg: the mixed-precision run of the logistic
    regression, tcgen05 gradient launches 1 (init) to 4; logreg_x3: the same with
    the three-term split form (LAPS_BF16X3); batch: 32 problems of the
    batch (d < 10^4, 33 M coordinates), batch_kernel launch 1 (init), 2 and 3 (5
    unadjusted iterations each); dense: the ill-conditioned Gaussian, gradient
    launches 1 (init) to 4."""
    import torch
    from paper_2601_16696_gb300 import build, laps, workloads
    build.build()
    info = {"ncu_case": which}
    if which in ("logreg", "logreg_x3"):
        pr = workloads.logreg()
        s = laps.Sampler(laps.Target.from_problem(pr), pr.M, n_total_steps=pr.n_steps,
                         precision=1 if which == "logreg" else 2)
        s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)
        s.step(3)
    elif which in ("batch", "batch_big", "batch_adj", "batch_big_adj"):
        if which.startswith("batch_big"):  # the batch's d = 10^4 problem on 4096 of its chains (330 MB)
            probs = [p for p in workloads.batch64() if p.d == 10000]
            probs[0].M = 4096
        else:
            probs = [p for p in workloads.batch64() if p.d < 10000][:32]
        adj = which.endswith("_adj")
        b = laps.Batch(probs, use_x0=False, n_total_steps=2000, **({"force_switch_at": 1} if adj else {}))
        b.set_shape(20, 0, 128)  # the shape the autotuner picks for the whole batch
        b.init(seed=0)
        if adj:
            b.step(1)  # launch 2: the first unadjusted step and the switch
            b.step(2)  # launch 3: two MAMS proposals of every problem
        else:
            b.step(5)  # launches 2 and 3: five unadjusted iterations each
            b.step(5)
        info.update(coordinates=sum(p.d * p.M for p in probs), shape=b.shape())
    else:
        pr = workloads.icg()
        s = laps.Sampler(laps.Target.from_problem(pr), pr.M, n_total_steps=pr.n_steps)
        s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)
        s.step(3)
    torch.cuda.synchronize()
    print(json.dumps(info))
    return 0


def ablations():
    """The paper's ablations on the synthetic stand-ins, one JSON object:
    - mams_only: the adjusted phase alone (switch forced after the first step,
      so the diagonal preconditioner comes from the first ensemble and the step
      size from the bisection) against LAPS (Table "mams");
    - fixed_step: the unadjusted phase at fixed step sizes, multiples of the
      adaptive run's final one, against the adaptive schedule (Fig. "stepsize");
    - chains: LAPS against the number of chains M (Fig. "chains").
    Reported per run: gradient evaluations per chain until b^2 < 0.01 (None
    if never), its wall time, and the final b^2."""
    import torch
    from paper_2601_16696_gb300 import build, laps, workloads
    build.build()
    torch.cuda.set_device(0)

    def go(pr, key, **cfg):
        tg = laps.Target.from_problem(pr)
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, stop_b2=0.01,
                         stop_b2_max=1 if key == "b2_max" else 0, **cfg)
        s.set_truth(pr.Ex2, pr.Varx2)
        s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=11)
        s.run()
        st = s.stats()
        hit = st["b2_first_t"] >= 0
        return {"grads_to_b2": st["b2_first_grads"] if hit else None,
                "ms_to_b2": st["b2_first_ns"] / 1e6 if hit else None,
                "t_switch": st["t_switch"], "final_" + key: st[key], "eps": st["eps"]}

    out = {"b2_threshold": 0.01, "seed": 11}
    mo = {}
    for name, pr, key in (("banana_d100_M4096", workloads.banana(), "b2_max"),
                          ("gauss_d100_M256", workloads.gauss_diag(), "b2_avg"),
                          ("icg_d100_M4096", workloads.icg(), "b2_max")):
        mo[name] = {"b2": key, "laps": go(pr, key), "mams_only": go(pr, key, force_switch_at=1)}
    out["mams_only"] = mo
    pr = workloads.gauss_diag()
    base = go(pr, "b2_avg", adjusted=0)
    ref = laps.Sampler(laps.Target.from_problem(pr), pr.M, n_total_steps=pr.n_steps)
    ref.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=11)
    ref.step(400)
    eps_end = ref.stats()["eps"]
    fs = {"workload": "gauss_d100_M256, unadjusted only", "b2": "b2_avg", "adaptive": base,
          "eps_adaptive_at_t400": eps_end}
    for f in (0.5, 1.0, 2.0, 4.0):
        fs["fixed_%gx" % f] = go(pr, "b2_avg", fixed_eps=f * eps_end, adjusted=0)
    out["fixed_step"] = fs
    ch = {"workload": "gauss_d100, 2000 steps", "b2": "b2_avg"}
    for M in (32, 64, 128, 256, 512, 1024, 4096):
        ch["M%d" % M] = go(workloads.gauss_diag(M=M), "b2_avg")
    out["chains"] = ch
    print(json.dumps(out))
    return 0


def ncu_case(adjusted: bool = False):
    import torch
    from paper_2601_16696_gb300 import build, laps, workloads
    build.build()
    pr = workloads.banana(d=RESIDENT["d"], M=RESIDENT["M"], n_steps=RESIDENT["n_steps"])
    tg = laps.Target.from_problem(pr)
    s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, force_switch_at=RESIDENT["switch_at"])
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)  # resident launch 1
    if adjusted:
        s.step(RESIDENT["switch_at"])                                         # launch 2: to the switch
        s.step(10)                                                            # launch 3: 10 proposals
    else:
        s.step(20)                                                            # resident launch 2
        s.step(200)                                                           # resident launch 3
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": pr.name, "t": s.stats()["t"], "launch": s.launch_info()}))
    return 0


def _resident_form(stream, seed0, peak, runs=5):
    """The register-resident form on the banana target (d = 100, M = 4096, 5000
    steps, switch forced at the first full window): whole-run throughput, time
    to b^2_max < 0.01, the kernel against its ALU roofline, and the same run
    end to end through the context API with host buffers."""
    import torch
    from paper_2601_16696_gb300 import laps, workloads
    pr = workloads.banana(d=RESIDENT["d"], M=RESIDENT["M"], n_steps=RESIDENT["n_steps"])
    tg = laps.Target.from_problem(pr)
    cfg = dict(n_total_steps=pr.n_steps, force_switch_at=RESIDENT["switch_at"])
    s = laps.Sampler(tg, pr.M, **cfg)
    s.set_truth(pr.Ex2, pr.Varx2)
    x0_dev = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    x0_host = torch.tensor(pr.x0, dtype=torch.float32).pin_memory()
    out_host = torch.empty(pr.M, pr.d, dtype=torch.float32).pin_memory()
    x0_e2e = torch.empty_like(x0_dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def timed(fn, n, sd0):
        ts, b2 = [], []
        for k in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(sd0 + k)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            st = s.stats()
            b2.append(st["b2_first_ns"] / 1e6 if st["b2_first_t"] >= 0 else None)
        return ts, b2

    def one(sd):
        s.init(x0_dev, seed=sd)
        s.run()

    for k in range(3):
        one(seed0 + k)
    ts, b2 = timed(one, runs, seed0 + 10)
    st = s.stats()
    grads = st["grads"]
    tr = s.trace()
    n_unadj = sum(1 for r in tr[1:] if r["phase"] == 0 or r["t"] == st["t_switch"])
    n_adj_grads = grads - 1 - n_unadj
    ms = statistics.mean(ts)
    info = s.launch_info()
    kern = "laps_resident_kernel<banana,%d,%d>" % (info["lanes_per_chain"], info["coords_per_lane"])
    ops = pr.M * pr.d * (n_unadj * ALU_OPS_LF + n_adj_grads * ALU_OPS_MN2_PER_GRAD)

    def e2e_run(sd):
        x0_e2e.copy_(x0_host, non_blocking=True)
        s.init(x0_e2e, seed=sd)
        s.run()
        s.sample(out=x0_e2e)
        out_host.copy_(x0_e2e, non_blocking=True)

    te, _ = timed(e2e_run, runs, seed0 + 20)
    # the kernel alone: events around laps_run (the initialisation is its own launch)
    k_ms = []
    for k in range(runs):
        s.init(x0_dev, seed=seed0 + 30 + k)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.run()
        b.record(stream)
        b.synchronize()
        k_ms.append(a.elapsed_time(b))
    kms = statistics.mean(k_ms)
    achieved = ops / (kms * 1e-3) / 1e9
    hits = [v for v in b2 if v is not None]
    n_prop = sum(1 for r in tr[1:] if r["phase"] == 1 and r["t"] != st["t_switch"])
    rec = _recorded(kern)  # [DRAM bytes per launch, warp instructions per coordinate: LF step, proposal]
    issue = None
    if rec and len(rec) >= 3:
        inst = pr.M * pr.d * (n_unadj * rec[1] + n_prop * rec[2])
        issue = {"frac": inst / (kms * 1e-3) / (peak * 1e9 / 32.0),
                 "warp_inst_per_coord": {"lf_step": rec[1], "proposal": rec[2]},
                 "basis": "ncu smsp__inst_executed of an unadjusted and an adjusted launch "
                          "(profiles/resident_traffic.txt) over the kernel time, against SMs x 4 "
                          "schedulers x 1 warp instruction per clock"}
    return {"workload": "%s_M%d_%dsteps" % (pr.name, pr.M, pr.n_steps),
            "switch": "after %d unadjusted steps (first full window)" % RESIDENT["switch_at"],
            "value": pr.M * grads / (ms * 1e-3), "unit": UNIT, "run_ms": ms, "runs": runs,
            "grads_per_chain": grads, "launch": info,
            "time_to_b2_ms": {"b2": "b2_max", "mean": statistics.mean(hits) if hits else None,
                              "reached": len(hits), "of": runs},
            "e2e": {"value": pr.M * grads / (statistics.mean(te) * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": x0_host.numel() * 4, "d2h_bytes_per_step": out_host.numel() * 4},
            "l2": "flushed (256 MB write) between runs",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                         "frac": achieved / peak, "traffic": _recorded_traffic(kern), "kernel": kern,
                         "kernel_ms": kms, "alu_ops": ops, "issue": issue}}


def _sharded_logreg(stream, world, rank, seed0, runs=2):
    """The chain-sharded ensemble (laps_create_sharded) on the logistic
    regression (d = 101, n = 10^4, M = 8192, mixed precision, 2000 steps): each
    rank advances M / N chains and exchanges its column totals once per
    iteration (an NCCL all-gather; a local copy on one rank).  Every rank calls
    this; the value counts all ranks' chains over the slowest rank's time."""
    import torch
    from paper_2601_16696_gb300 import laps, workloads
    pr = workloads.logreg()
    tg = laps.Target.from_problem(pr)
    m0, m1 = rank * pr.M // world, (rank + 1) * pr.M // world
    fn = laps.nccl_allgather() if world > 1 else None
    s = laps.Sampler(tg, m1 - m0, n_total_steps=pr.n_steps, precision=1,
                     shard=(pr.M, m0, rank, world, fn))
    x0 = torch.tensor(pr.x0[m0:m1], dtype=torch.float32, device="cuda")
    one = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, precision=1) if world == 1 else None
    x0_all = torch.tensor(pr.x0, dtype=torch.float32, device="cuda") if world == 1 else None

    def timed(smp, x, sd):
        smp.init(x, seed=sd)
        smp.step(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        smp.init(x, seed=sd + 1)
        smp.run()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    ts = [timed(s, x0, seed0 + 2 * k) for k in range(runs)]
    ms = _max_over_ranks(min(ts))
    st = s.stats()
    out = {"workload": "logreg_d%d_n%d_M%d_%dsteps, mixed precision, %d rank(s) of %d chains"
                       % (pr.d, pr.X.shape[0], pr.M, pr.n_steps, world, m1 - m0),
           "value": pr.M * st["grads"] / (ms * 1e-3), "unit": UNIT, "run_ms": ms,
           "grads_per_chain": st["grads"], "t": st["t"],
           "exchange": "NCCL all-gather of 4 d_pad + 5 float-float pairs per rank and iteration"
                       if world > 1 else "one rank: a local copy of its totals"}
    if one is not None:
        out["unsharded_run_ms"] = min(timed(one, x0_all, seed0 + 10 + 2 * k) for k in range(runs))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="laps", choices=["laps", "reference"])
    ap.add_argument("--partition", default="replicas", choices=["replicas", "problems"],
                    help="N > 1: every rank runs the whole batch (replicas, weak scaling) or its "
                         "share of the batch's problems (laps_batch_partition, strong scaling)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="runs timed end to end (default: a quarter of --steps, at least 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other forms (resident, logistic regression, ...)")
    ap.add_argument("--ncu-case", action="store_true",
                    help="no timing: the resident workload's launch shape, one launch of 200 "
                         "unadjusted iterations after two others (the case profiled under ncu)")
    ap.add_argument("--ncu-case-adjusted", action="store_true",
                    help="no timing: as --ncu-case, the third launch runs 10 MAMS proposals")
    ap.add_argument("--ncu-case-form", choices=["logreg", "logreg_x3", "batch", "batch_big", "batch_adj",
                                                "batch_big_adj", "dense"],
                    help="no timing: a small case of another kernel (for ncu)")
    ap.add_argument("--ablations", action="store_true",
                    help="no contract line: the paper's ablations (MAMS only, fixed step, "
                         "number of chains) as one JSON object")
    args = ap.parse_args()
    if args.ablations:
        return ablations()
    if args.ncu_case_form:
        return ncu_case_form(args.ncu_case_form)
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case or args.ncu_case_adjusted:
        return ncu_case(adjusted=args.ncu_case_adjusted)

    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2601_16696_gb300 import build, laps, workloads
    build.build()
    stream = torch.cuda.current_stream()
    seed_base = 1000 * rank
    K_ipl = BATCH["iters_per_launch"]

    # ---- the batch: initial positions in one device buffer (one H2D copy for e2e)
    all_probs = workloads.batch64(n_steps=BATCH["n_steps"])
    by_problems = args.partition == "problems" and world > 1
    if by_problems:
        # this rank's share; the problems keep their Philox ids of the whole batch
        ids = laps.partition_problems(all_probs, world)[rank]
        if not ids:
            raise SystemExit("--partition problems: rank %d owns no problem (%d ranks, %d problems)"
                             % (rank, world, len(all_probs)))
        seed_base = 0
    else:
        ids = list(range(len(all_probs)))
    probs = [all_probs[k] for k in ids]
    sizes = [p.M * p.d for p in probs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    total = int(offs[-1])
    x0_host = torch.empty(total, dtype=torch.float32).pin_memory()
    for p, o in zip(probs, offs):
        x0_host[int(o):int(o) + p.M * p.d].copy_(torch.from_numpy(p.x0.astype(np.float32).ravel()))
    x0_dev = x0_host.cuda()
    out_dev = torch.empty(total, dtype=torch.float32, device="cuda")
    out_host = torch.empty(total, dtype=torch.float32).pin_memory()
    views = [dataclasses.replace(p, x0=x0_dev[int(o):int(o) + p.M * p.d].view(p.M, p.d))
             for p, o in zip(probs, offs)]
    outs = [out_dev[int(o):int(o) + p.M * p.d].view(p.M, p.d) for p, o in zip(probs, offs)]
    b = laps.Batch(views, n_total_steps=BATCH["n_steps"], force_switch_at=BATCH["switch_at"], ids=ids)
    for k, p in enumerate(probs):
        b.set_truth(k, p.Ex2, p.Varx2)
    b.init(seed=seed_base)
    b.tune()
    n = len(probs)

    def one_run(sd):
        b.init(seed=sd)
        b.run(iters_per_launch=K_ipl)

    def e2e_run(sd):
        x0_dev.copy_(x0_host, non_blocking=True)
        b.init(seed=sd)
        b.run(iters_per_launch=K_ipl)
        for k in range(n):
            b.sample(k, out=outs[k])
        out_host.copy_(out_dev, non_blocking=True)

    def timed(fn, steps, sd0):
        ts, b2 = [], []
        for k in range(steps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(sd0 + k)
            e.record(stream)
            e.synchronize()
            ts.append(a.elapsed_time(e))
            sts = [b.stats(q) for q in range(n)]
            b2.append(max(st["b2_first_ns"] / 1e6 if st["b2_first_t"] >= 0 else math.inf for st in sts))
        return ts, b2, sts

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    for k in range(args.warmup):
        one_run(seed_base + k)
    torch.cuda.synchronize()

    # ---- device-resident timing (the headline value)
    barrier()
    with Clocks(local) as clk:
        ts, b2, sts = timed(one_run, args.steps, seed_base + 100)
    barrier()
    assert all(st["done"] for st in sts), "a problem did not finish"
    chain_grads = sum(p.M * st["grads"] for p, st in zip(probs, sts))
    # the units every rank processed: replicas run the whole batch each, a
    # partition's ranks their shares of one batch
    job_grads = _sum_over_ranks(float(chain_grads))
    ms = _max_over_ranks(statistics.mean(ts))
    value = job_grads / (ms * 1e-3)
    clocks = clk.summary()

    # ---- end to end through the batch entry points with host buffers
    n_e2e = args.e2e_steps or max(2, args.steps // 4)
    barrier()
    te, _, _ = timed(e2e_run, n_e2e, seed_base + 200)
    barrier()
    e2e_ms = _max_over_ranks(statistics.mean(te))
    e2e = {"value": job_grads / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": x0_host.numel() * 4, "d2h_bytes_per_step": out_host.numel() * 4,
           "ms_per_step": e2e_ms, "steps": n_e2e}

    # ---- the kernel's own duration: CUDA events around every launch of one run
    b.init(seed=seed_base + 300)
    kev = []
    iters_max = BATCH["n_steps"] + 1
    for r in range(iters_max // K_ipl + 2):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.step(K_ipl)
        e.record(stream)
        kev.append((a, e))
    torch.cuda.synchronize()
    launch_ms = [a.elapsed_time(e) for a, e in kev]
    ksts = [b.stats(q) for q in range(n)]
    live = [x for x in launch_ms if x > 0.05]  # launches after every problem finished return at once
    kms = sum(live)
    ops, hbm = 0.0, 0.0
    n_unadj = {}
    for k, (p, st) in enumerate(zip(probs, ksts)):
        tr = b.trace(k)
        nu = sum(1 for r in tr[1:] if r["phase"] == 0 or r["t"] == st["t_switch"])
        npr = len(tr) - 1 - nu
        n_unadj[k] = nu
        # a proposal: the full velocity refresh (an O map's noise) and N steps
        per_prop = OPS_O + 15 * BATCH_OPS_STEP[st["integrator"]] if st["integrator"] else 0.0
        ops += p.M * p.d * (nu * BATCH_OPS_LF + npr * per_prop)
        hbm += p.M * p.d * 16.0 * (nu + npr)  # y, u read and written once per iteration
    mhz = clocks["sm_mhz"] or 1455.0
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = nsm * 128 * mhz * 1e6 / 1e9  # FP32-pipe lane issue rate, Gop/s
    achieved = ops / (kms * 1e-3) / 1e9
    pk = _peaks()
    sh = b.shape()
    kern = "batch_kernel<%d>" % sh["coords_per_lane"]
    rec = _recorded(kern, "batch_counters.txt", BATCH_SRC)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                "frac": achieved / peak, "traffic": None, "kernel": kern, "kernel_ms": kms,
                "launches": len(live),
                "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (measured median)" % (nsm, mhz),
                "hbm": {"achieved_gbs": hbm / (kms * 1e-3) / 1e9, "peak_gbs": pk["hbm_gbs"],
                        "frac": hbm / (kms * 1e-3) / 1e9 / pk["hbm_gbs"],
                        "basis": "16 B per coordinate and iteration (y, u read and written)"}}
    if rec and len(rec) >= 4:
        # [DRAM bytes per coordinate: LF step; warp instructions per coordinate: LF step,
        # proposal; DRAM bytes per coordinate: proposal] from ncu captures of the batch's
        # parts, scaled by a run's work and averaged over its launches
        bytes_run = sum(p.M * p.d * (rec[0] * n_unadj[k] + rec[3] * (len(b.trace(k)) - 1 - n_unadj[k]))
                        for k, p in enumerate(probs))
        roofline["traffic"] = bytes_run / len(live)
        inst = sum(p.M * p.d * (rec[1] * n_unadj[k] + rec[2] * (len(b.trace(k)) - 1 - n_unadj[k]))
                   for k, p in enumerate(probs))
        roofline["issue"] = {"warp_inst_per_coord": {"lf_step": rec[1], "proposal": rec[2]},
                             "frac": inst / (kms * 1e-3) / (nsm * 4 * mhz * 1e6),
                             "basis": "ncu smsp__inst_executed of unadjusted and adjusted launches of the "
                                      "batch's parts (profiles/batch_counters.txt); peak %d SMs x 4 "
                                      "schedulers x 1 warp instruction per clock" % nsm}

    # every rank draws from the same seed: the ranks hold parts of one ensemble
    sharded = None if args.no_forms else _sharded_logreg(stream, world, rank, 600)

    if rank == 0:
        reached = [v for v in b2 if v < math.inf]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if by_problems else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _batch_config(all_probs),
            "run": {"chain_grads_per_run": job_grads if by_problems else chain_grads, "shape": sh,
                    "iters_per_launch": K_ipl,
                    "integrators": sorted({("MN4" if st["integrator"] == 2 else "MN2") for st in sts}),
                    "parallelism": ("problems over %d ranks (laps_batch_partition; rank 0 runs %d of %d)"
                                    % (world, len(probs), len(all_probs))) if by_problems
                                   else "replicas" if world > 1 else "1 GPU"},
            "time_to_b2": {"ms": statistics.mean(reached) if reached else None, "b2": "b2_avg",
                           "threshold": 0.01, "over": "every problem", "runs_reached": len(reached),
                           "of": len(b2)},
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": args.steps * (2 + BATCH["n_steps"] // K_ipl + 2),
            "clocks": clocks,
        }
        if not args.no_forms:
            forms = {"resident": _resident_form(stream, seed_base + 400, peak)}
            forms.update(_forms(torch.empty(256 << 20, dtype=torch.uint8, device="cuda"), stream, mhz,
                                seed_base + 500))
            forms["logreg_sharded"] = sharded
            line["forms"] = forms
            line["measured_peaks"] = _probe_peaks(stream)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _batch_oracle(all_probs, total_chain_grads=job_grads if by_problems
                                                 else chain_grads, iters=12)
            if not args.no_forms:
                line["cpu_baseline"]["other_workloads"] = _oracle_rates()
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
