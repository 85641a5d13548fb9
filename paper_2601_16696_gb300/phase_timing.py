"""Per-phase device time of one block of the register-resident kernel (a
diagnostic build, not the product library).

    python -m paper_2601_16696_gb300.phase_timing [block]

builds the library with -DLAPS_PHASE_TIMING (and LAPS_PHASE_BLOCK = block,
default 0) into liblaps_phase<block>.so beside the product library, runs the
banana workload (d = 100, M = 4096) for 500 unadjusted iterations at a fixed
step, 500 with the step-size controller, and 40 MAMS proposals after a switch
at step 1000, and prints the mean microseconds per iteration between the
kernel's phase marks (the marks synchronise the block, so the sum is not
exactly the undisturbed iteration).
"""
import ctypes as C
import os
import sys

import numpy as np
import torch

from . import build, laps, workloads

PHASES = ["chain update", "block columns", "chain sums", "barrier 1", "slice", "barrier 2",
          "gather+finalise"]


def main(block: int = 0) -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblaps_phase%d.so" % block)
    path = build.build(extra_flags=("-DLAPS_PHASE_TIMING", "-DLAPS_PHASE_BLOCK=%d" % block), out=out)
    L = laps.lib(path)
    L.laps_debug_phase_ns.argtypes = [C.c_void_p, C.POINTER(C.c_ulonglong)]
    L.laps_debug_phase_ns.restype = C.c_int
    pr = workloads.banana()
    tg = laps.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    for label, cfg, warm, n in (("unadjusted, fixed step", dict(fixed_eps=0.05), 20, 500),
                                ("unadjusted, adaptive step", dict(adjusted=0), 20, 500),
                                ("adjusted, switch at step 1000", dict(force_switch_at=1000), 1010, 40)):
        s = laps.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
        L.laps_debug_phase_ns(s._h, None)
        s.init(x0, seed=0)
        s.step(warm)
        buf = (C.c_ulonglong * 16)()
        L.laps_debug_phase_ns(s._h, buf)  # read and reset
        s.step(n)
        L.laps_debug_phase_ns(s._h, buf)
        v = np.array(list(buf), dtype=np.float64) / n / 1e3
        print("block %d, %s (phase %d), us per iteration: %s | total %.2f"
              % (block, label, s.stats()["phase"],
                 ", ".join("%s %.2f" % (nm, v[k]) for k, nm in enumerate(PHASES)), v[:7].sum()))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
