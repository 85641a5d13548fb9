"""Several live contexts at once.  A kernel's dynamic shared-memory limit is a
process-wide attribute, so a context created later with a smaller footprint
must not make an earlier, larger one's launches fail."""
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


def _x0(pr):
    return torch.tensor(pr.x0, dtype=torch.float32, device="cuda")


def test_streamed_contexts_of_different_size(L):
    big = W.logreg(n_data=500, n_feat=100, M=256, n_steps=50)   # d_pad 128
    small = W.logreg(n_data=500, n_feat=20, M=256, n_steps=50)  # d_pad 64: same seg kernel, less memory
    tb, ts = L.Target.from_problem(big), L.Target.from_problem(small)
    sb = L.Sampler(tb, big.M, n_total_steps=big.n_steps)
    ss = L.Sampler(ts, small.M, n_total_steps=small.n_steps)
    sb.init(_x0(big), seed=0)
    sb.step(3)
    ss.init(_x0(small), seed=0)
    ss.step(3)
    assert sb.stats()["t"] == 3 and ss.stats()["t"] == 3


def test_resident_contexts_of_different_size(L):
    big = W.banana(d=100, M=512, n_steps=50)
    small = W.banana(d=20, M=512, n_steps=50)
    sb = L.Sampler(L.Target.from_problem(big), big.M, n_total_steps=big.n_steps,
                   lanes_per_chain=16, coords_per_lane=8)
    ss = L.Sampler(L.Target.from_problem(small), small.M, n_total_steps=small.n_steps,
                   lanes_per_chain=16, coords_per_lane=8)
    assert sb.launch_info()["resident"] == 1 == ss.launch_info()["resident"]
    sb.init(_x0(big), seed=0)
    sb.step(3)
    ss.init(_x0(small), seed=0)
    ss.step(3)
    assert sb.stats()["t"] == 3 and ss.stats()["t"] == 3
    assert np.isfinite(sb.sample().cpu().numpy()).all()
