"""The stream contract of include/laps.h: the calls it lists as enqueue-only
return before their GPU work ends.

laps_init and a long laps_step of the register-resident path, laps_batch_init
and laps_batch_run enqueue work and return; the stream is still busy when
they do (cudaStreamQuery reports not ready), and the results read afterwards
equal those of runs that were waited for step by step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_16696_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16696_gb300 import build, laps
    build.build()
    laps.lib()
    return laps


def test_resident_init_and_step_only_enqueue(L):
    pr = W.banana(d=100, M=4096, n_steps=5000)
    tg = L.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ref = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps)
    ref.init(x0, seed=4)
    torch.cuda.synchronize()
    for _ in range(10):
        ref.step(100)
        torch.cuda.synchronize()
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps)
    torch.cuda.synchronize()
    s.init(x0, seed=4)
    s.step(1000)  # ~13 ms of device work
    pending = not stream.query()
    torch.cuda.synchronize()
    assert pending
    np.testing.assert_array_equal(s.sample().cpu().numpy(), ref.sample().cpu().numpy())
    assert s.stats()["t"] == ref.stats()["t"] == 1000


def test_batch_init_and_run_only_enqueue(L):
    probs = [W.gauss_diag(d=d, M=M, n_steps=400, x0_scale=1.0, var_lo=0.1, var_hi=10.0, seed=50 + k)
             for k, (d, M) in enumerate([(40, 512), (300, 1024), (2000, 512)])]
    stream = torch.cuda.current_stream()
    ref = L.Batch(probs, n_total_steps=400, force_switch_at=150)
    ref.init(seed=8)
    torch.cuda.synchronize()
    for _ in range(600):
        ref.step(1)
    torch.cuda.synchronize()
    b = L.Batch(probs, n_total_steps=400, force_switch_at=150)
    torch.cuda.synchronize()
    b.init(seed=8)
    b.run(iters_per_launch=32)
    pending = not stream.query()
    torch.cuda.synchronize()
    assert pending
    for k in range(len(probs)):
        st, sr = b.stats(k), ref.stats(k)
        # 150 unadjusted steps, then 16 proposals of 15 steps (a 17th would pass 400)
        assert st["done"] == sr["done"] == 1 and st["t"] == sr["t"] == 390
        np.testing.assert_array_equal(b.sample(k).cpu().numpy(), ref.sample(k).cpu().numpy())
