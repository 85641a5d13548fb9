"""The allocation-free entry point, laps_run_noalloc, through the C ABI.

It serves callers that cannot call cudaMalloc (a process whose device memory
belongs to a pool allocator that reserved the GPU, code that must not add the
synchronisation cudaMalloc implies, a plug-in that may not grow the device
footprint): the run's scratch lives in a fixed array inside the library,
shared by every call.  Two calls in a row, on different problems, must each
give what the context API (laps_create / laps_init / laps_run /
laps_sample) gives for the same inputs and random stream.
"""
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


def _context_api(L, pr, seed, cfg):
    tg = L.Target.from_problem(pr)
    s = L.Sampler(tg, pr.M, **cfg)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=seed)
    s.run()
    return s.sample(), s.stats()


def test_noalloc_matches_context_api_on_two_calls(L):
    cases = [
        (W.banana(d=20, M=1000, n_steps=400), dict(n_total_steps=400, force_switch_at=150), 5),
        (W.gauss_diag(d=100, M=256, n_steps=300), dict(n_total_steps=300, force_switch_at=100), 7),
    ]
    for pr, cfg, seed in cases:
        ref, st_ref = _context_api(L, pr, seed, cfg)
        x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
        prec = (torch.tensor(pr.prec, dtype=torch.float32, device="cuda")
                if pr.prec is not None else None)
        out = torch.full_like(ref, float("nan"))
        st = L.run_noalloc(pr.kind, pr.d, pr.M, x0, seed, out, prec=prec,
                           banana_sb=pr.banana_sb, funnel_sv=pr.funnel_sv, **cfg)
        rel = ((out - ref).norm(dim=1) / ref.norm(dim=1)).max().item()
        assert rel <= 1e-5, rel
        assert (st["t"], st["grads"], st["phase"], st["t_switch"]) == \
            (st_ref["t"], st_ref["grads"], st_ref["phase"], st_ref["t_switch"])
        assert st["eps"] == pytest.approx(st_ref["eps"], rel=1e-5)


def test_noalloc_rejects_problems_beyond_its_array(L):
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LapsError) as err:
        # 200000 steps: the moving window alone (T = 40000 rows of d = 100) needs 32 MB
        L.run_noalloc(L.BANANA, 100, 256, None, 0, out, n_total_steps=200000)
    assert err.value.status == 1 and "bytes of scratch" in str(err.value)
