"""The C ABI (CPU-only checks): the library builds and loads, exports every
function include/laps.h declares, and the binding's struct layouts match the
C compiler's."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "laps.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(laps_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2601_16696_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (laps_\w+)", out))
    missing = [f for f in _declared() if f not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    from paper_2601_16696_gb300 import laps
    assert sorted(laps.SIGNATURES) == _declared()
    L = laps.lib(built)  # loads without a GPU
    for name in laps.SIGNATURES:
        assert hasattr(L, name)
    assert b"sm_103a" in L.laps_version()


def test_struct_layouts_match_c(tmp_path):
    from paper_2601_16696_gb300 import laps
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "laps.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d %d %d %d\\n",'
                    'sizeof(laps_config), sizeof(laps_stats), sizeof(laps_trace_row),'
                    'sizeof(laps_target_desc), sizeof(laps_launch_info),'
                    'offsetof(laps_config, barrier_extra_arrivals),'
                    'offsetof(laps_stats, b2_first_ns), sizeof(laps_problem),'
                    'offsetof(laps_problem, x0_scale), sizeof(laps_batch_shape),'
                    'sizeof(laps_peaks), offsetof(laps_peaks, grid_barrier_us),'
                    'sizeof(laps_shard), offsetof(laps_shard, user_data),'
                    '(int)LAPS_FP32, (int)LAPS_MIXED, (int)LAPS_BF16X3, (int)LAPS_MIXED_BF16X3);return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HDR), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    import ctypes as C
    want = [C.sizeof(laps.Config), C.sizeof(laps.Stats), C.sizeof(laps.TraceRow),
            C.sizeof(laps.TargetDesc), C.sizeof(laps.LaunchInfo),
            laps.Config.barrier_extra_arrivals.offset, laps.Stats.b2_first_ns.offset,
            C.sizeof(laps.Problem), laps.Problem.x0_scale.offset, C.sizeof(laps.BatchShape),
            C.sizeof(laps.Peaks), laps.Peaks.grid_barrier_us.offset,
            C.sizeof(laps.ShardSpec), laps.ShardSpec.user_data.offset,
            laps.FP32, laps.MIXED, laps.BF16X3, laps.MIXED_BF16X3]
    assert got == want


def test_config_defaults_are_the_papers(built):
    from paper_2601_16696_gb300 import laps
    c = laps.default_config()
    assert (c.C, c.alpha, c.switch_tol, c.window_frac, c.acc_tol, c.adj_L_factor) == \
        (0.025, 2.0, 0.01, 0.2, 0.03, 1.25)
    assert (c.steps_per_proposal, c.mn4_min_dim, c.a_target_mn2, c.a_target_mn4, c.eps0_coef) == \
        (15, 200, 0.7, 0.9, 0.01)
