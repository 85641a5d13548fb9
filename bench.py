"""Benchmark of the LAPS hot path on GB300: one JSON line on stdout.

A step is one complete LAPS run (Algorithm 1: initialisation, the unadjusted
phase, the switch, the adjusted phase, the samples) of the workload: the
banana target, d = 100, M = 4096 chains, 5000 integrator steps.  The paper's
default switch rule would keep this ensemble unadjusted (its window statistic
stays above 0.01 at M = 4096), so the timed runs switch after the first window
(1000 steps, the paper's "number of unadjusted steps" ablation knob) and run
MAMS proposals for the remaining 4000 steps.

value      chain-gradient-evals/s = M x gradient evaluations per chain / time,
           inputs resident on the device, CUDA events on the launching stream.
e2e        the same metric through the public API with host buffers: x0 copied
           from pinned host memory and the samples copied back in the timed
           region.
time_to_b2 wall time (CUDA events) of runs that stop at b^2_max < 0.01.
roofline   the persistent kernel against the FP32 ALU issue rate: algorithmic
           operations of the run (the per-coordinate counts below) over the
           kernel's own duration, against SMs x 128 lanes x the measured clock.
cpu_baseline  the FP64 oracle on the host cores on a bounded sample.

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
WORKLOAD = dict(name="banana_d100", d=100, M=4096, n_steps=5000, switch_at=1000)
# algorithmic ALU operations per coordinate and gradient evaluation: an LF
# unadjusted step (two O maps: a quarter Philox4x32-10 call, half a Box-Muller
# pair, uniforms and the O arithmetic, 48 each; two B maps, the A map with the
# target and the ensemble sums, 21) and an MN2 adjusted step per gradient
ALU_OPS_LF = 117.0
ALU_OPS_MN2_PER_GRAD = 61.0


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


def _kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_16696_gb300", "csrc")
    for f in ("laps_resident_kernel.cuh", "laps_resident.cuh", "laps_finalise.cuh", "laps_device.cuh",
              "laps_params.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel: str):
    """DRAM bytes per launch from the ncu capture in profiles/, or None when the
    kernel sources changed after that capture."""
    path = os.path.join(ROOT, "profiles", "resident_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = _kernel_source_hash()
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == cur:
            return float(f[2])
    return None


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


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    from paper_2601_16696_gb300 import workloads
    pr = workloads.banana(d=WORKLOAD["d"], M=WORKLOAD["M"], n_steps=WORKLOAD["n_steps"])
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(_cpu_baseline(pr))
    timed = vals[args.warmup:]
    v = statistics.mean(r["value"] for r in timed)
    ms = statistics.mean(1e3 * pr.M * 500 / r["value"] for r in timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%s_M%d_%dsteps" % (pr.name, pr.M, pr.n_steps),
                       "switch": "after %d unadjusted steps (first full window)" % WORKLOAD["switch_at"],
                       "parallelism": "host cores (the oracle)"},
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
    unadjusted phase beside the all-FP32 form; the batch of 64 uneven diagonal
    Gaussians plus one d = 10^4, M = 16384 problem in one persistent launch; the
    rotated ill-conditioned Gaussian (d = 100, M = 4096, dense precision).
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
    tg = laps.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    n = pr.X.shape[0]
    flops = 4.0 * pr.M * n * pr.d  # Z = W X^T and G = R X per gradient of the ensemble
    lr = {"workload": "logreg_d%d_n%d_M%d_%dsteps" % (pr.d, n, pr.M, pr.n_steps),
          "b2": "b2_max", "truth": "Laplace approximation of the posterior (FP64)",
          "switch": "paper rule (max delta < 0.01)"}
    kernels = {0: "logreg_grad_f32_kernel<128>", 1: "logreg_grad_mma_kernel<128>",
               2: "logreg_grad_x3_kernel<128>"}
    for name, prec in (("mixed", 1), ("fp32", 0), ("bf16x3", 2)):
        for _ in range(3):
            tg.logp_grad(x0, precision=prec)
        reps = 10
        gms = timed_ms(lambda: [tg.logp_grad(x0, precision=prec) for _ in range(reps)]) / reps
        tg.check()
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, precision=prec, stop_b2=0.01,
                         stop_b2_max=1)
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
    # ---- the batch
    probs = workloads.batch64()
    coords = sum(p.d * p.M for p in probs)
    b = laps.Batch(probs, use_x0=False, n_total_steps=2000)
    for k, p in enumerate(probs):
        b.set_truth(k, p.Ex2, p.Varx2)
    b.init(seed=seed0)
    b.tune()
    b.step(2)
    it_ms = timed_ms(lambda: b.step(5)) / 5  # unadjusted iterations of every problem
    b.init(seed=seed0 + 1)
    run_ms = timed_ms(lambda: b.run(iters_per_launch=64))
    sts = [b.stats(k) for k in range(len(probs))]
    grads = sum(p.M * s["grads"] for p, s in zip(probs, sts))
    firsts = [s["b2_first_ns"] / 1e6 for s in sts if s["b2_first_t"] >= 0]
    achieved = coords * 16 / (it_ms * 1e-3) / 1e9
    out["batch"] = {
        "workload": "batch64: 64 Gaussians d in [10, 2000], M in {512..4096}, "
                    "+ d=10000 M=16384; 2000 steps, paper switch rule",
        "problems": len(probs), "coordinates": coords,
        "value": grads / (run_ms * 1e-3), "unit": UNIT, "run_ms": run_ms,
        "time_to_b2_ms": {"b2": "b2_avg", "reached": len(firsts), "of": len(probs),
                          "max": max(firsts) if firsts else None,
                          "median": statistics.median(firsts) if firsts else None},
        "shape": b.shape(),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": None,
                     "kernel": "batch_kernel<%d>" % b.shape()["coords_per_lane"],
                     "basis": "16 B per coordinate-step (y, u read and written), %.3f ms per "
                              "unadjusted iteration of the whole batch" % it_ms},
    }
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
    elif which == "batch":
        probs = [p for p in workloads.batch64() if p.d < 10000][:32]
        b = laps.Batch(probs, use_x0=False, n_total_steps=2000)
        b.init(seed=0)
        b.step(5)
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
    pr = workloads.banana(d=WORKLOAD["d"], M=WORKLOAD["M"], n_steps=WORKLOAD["n_steps"])
    tg = laps.Target.from_problem(pr)
    s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, force_switch_at=WORKLOAD["switch_at"])
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)  # resident launch 1
    if adjusted:
        s.step(WORKLOAD["switch_at"])                                         # launch 2: to the switch
        s.step(10)                                                            # launch 3: 10 proposals
    else:
        s.step(20)                                                            # resident launch 2
        s.step(200)                                                           # resident launch 3
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": pr.name, "t": s.stats()["t"], "launch": s.launch_info()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="laps", choices=["laps", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the logistic-regression and batch forms")
    ap.add_argument("--ncu-case", action="store_true",
                    help="no timing: the workload's launch shape, one launch of 200 unadjusted "
                         "iterations after two others (the case profiled under ncu)")
    ap.add_argument("--ncu-case-adjusted", action="store_true",
                    help="no timing: as --ncu-case, the third launch runs 10 MAMS proposals")
    ap.add_argument("--ncu-case-form", choices=["logreg", "logreg_x3", "batch", "dense"],
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

    pr = workloads.banana(d=WORKLOAD["d"], M=WORKLOAD["M"], n_steps=WORKLOAD["n_steps"])
    tg = laps.Target.from_problem(pr)
    cfg = dict(n_total_steps=pr.n_steps, force_switch_at=WORKLOAD["switch_at"])
    sampler = laps.Sampler(tg, pr.M, **cfg)
    sampler.set_truth(pr.Ex2, pr.Varx2)
    stopper = laps.Sampler(tg, pr.M, stop_b2=0.01, stop_b2_max=1, **cfg)
    stopper.set_truth(pr.Ex2, pr.Varx2)
    x0_dev = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    x0_host = torch.tensor(pr.x0, dtype=torch.float32).pin_memory()
    out_host = torch.empty(pr.M, pr.d, dtype=torch.float32).pin_memory()
    x0_e2e = torch.empty_like(x0_dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()
    seed_base = 1000 * rank

    def one_run(s, seed):
        s.init(x0_dev, seed=seed)
        s.run()

    def timed(fn, n, seed0):
        ts = []
        for k in range(n):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(seed0 + k)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    # ---- warm-up
    for k in range(args.warmup):
        one_run(sampler, seed_base + k)
        one_run(stopper, seed_base + k)
    torch.cuda.synchronize()
    st = sampler.stats()
    grads = st["grads"]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing (the headline value)
    barrier()
    with Clocks(local) as clk:
        ts = timed(lambda sd: one_run(sampler, sd), args.steps, seed_base + 100)
    barrier()
    st = sampler.stats()
    assert st["done"] and st["grads"] == grads, st
    ms = _max_over_ranks(statistics.mean(ts))
    value = world * pr.M * grads / (ms * 1e-3)

    # ---- the kernel's own duration and its ALU roofline
    info = sampler.launch_info()
    tr = sampler.trace()
    n_unadj = sum(1 for r in tr[1:] if r["phase"] == 0)
    n_adj_grads = grads - 1 - n_unadj
    k_ms = []
    for k in range(args.steps):
        sampler.init(x0_dev, seed=seed_base + 200 + k)
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sampler.run()
        b.record(stream)
        b.synchronize()
        k_ms.append(a.elapsed_time(b))
    kms = statistics.mean(k_ms)
    coord = pr.M * pr.d
    ops = coord * (n_unadj * ALU_OPS_LF + n_adj_grads * ALU_OPS_MN2_PER_GRAD)
    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or 1455.0
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = nsm * 128 * mhz * 1e6 / 1e9  # FP32-pipe lane issue rate, Gop/s
    achieved = ops / (kms * 1e-3) / 1e9
    traffic = _recorded_traffic("laps_resident_kernel<banana,%d,%d>"
                                % (info["lanes_per_chain"], info["coords_per_lane"]))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "laps_resident_kernel<banana,%d,%d>" % (info["lanes_per_chain"],
                                                                   info["coords_per_lane"]),
                "kernel_ms": kms,
                "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (measured median)" % (nsm, mhz)}

    # ---- wall time to b^2_max < 0.01
    t2 = timed(lambda sd: one_run(stopper, sd), args.steps, seed_base + 300)
    s2 = stopper.stats()
    time_to_b2 = {"ms": statistics.mean(t2), "b2": "b2_max", "threshold": 0.01,
                  "reached": s2["b2_max"] < 0.01, "t": s2["t"], "grads_per_chain": s2["grads"],
                  "phase_at_stop": s2["phase"]}

    # ---- end to end through the public API with host buffers
    def e2e_run(seed):
        x0_e2e.copy_(x0_host, non_blocking=True)
        sampler.init(x0_e2e, seed=seed)
        sampler.run()
        sampler.sample(out=x0_e2e)
        out_host.copy_(x0_e2e, non_blocking=True)

    te = timed(e2e_run, args.steps, seed_base + 400)
    e2e_ms = _max_over_ranks(statistics.mean(te))
    e2e = {"value": world * pr.M * grads / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": x0_host.numel() * 4, "d2h_bytes_per_step": out_host.numel() * 4,
           "ms_per_step": e2e_ms}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s_M%d_%dsteps" % (pr.name, pr.M, pr.n_steps),
                       "switch": "after %d unadjusted steps (first full window)"
                                 % WORKLOAD["switch_at"],
                       "grads_per_chain": grads, "l2": "flushed (256 MB write) between runs",
                       "launch": info, "parallelism": "replicas" if world > 1 else "1 GPU"},
            "time_to_b2": time_to_b2, "roofline": roofline, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "clocks": clocks,
        }
        if not args.no_forms:
            line["forms"] = _forms(flush, stream, mhz, seed_base + 500)
            line["measured_peaks"] = _probe_peaks(stream)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(pr, single_thread=True,
                                                 grads_to_b2=time_to_b2.get("grads_per_chain"))
            if not args.no_forms:
                line["cpu_baseline"]["other_workloads"] = _oracle_rates()
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
