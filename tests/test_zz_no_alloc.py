"""The allocation-free entry point, laps_run_noalloc, through the C ABI.

It serves callers that cannot call cudaMalloc (a process whose device memory
belongs to a pool allocator that reserved the GPU, code that must not add the
synchronisation cudaMalloc implies, a plug-in that may not grow the device
footprint): the run's scratch lives in a fixed array inside the library,
shared by every call.  Two calls in a row, on different problems, must each
give what the context API (laps_create / laps_init / laps_run /
laps_sample) gives for the same inputs and random stream: both run the same
kernel in the same launch shape on the same inputs, so bit for bit.  Once the
array is loaded, a call must leave the device's free memory unchanged.
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


CASES = [
    (W.banana(d=20, M=1000, n_steps=400), dict(n_total_steps=400, force_switch_at=150), 5),
    (W.gauss_diag(d=100, M=256, n_steps=300), dict(n_total_steps=300, force_switch_at=100), 7),
]


def _inputs(pr):
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    prec = torch.tensor(pr.prec, dtype=torch.float32, device="cuda") if pr.prec is not None else None
    return x0, prec


def test_noalloc_matches_context_api_on_two_calls(L):
    for pr, cfg, seed in CASES:
        ref, st_ref = _context_api(L, pr, seed, cfg)
        x0, prec = _inputs(pr)
        out = torch.full_like(ref, float("nan"))
        st = L.run_noalloc(pr.kind, pr.d, pr.M, x0, seed, out, prec=prec,
                           banana_sb=pr.banana_sb, funnel_sv=pr.funnel_sv, **cfg)
        assert torch.equal(out, ref), ((out - ref).abs().max().item())
        assert (st["t"], st["grads"], st["phase"], st["t_switch"]) == \
            (st_ref["t"], st_ref["grads"], st_ref["phase"], st_ref["t_switch"])
        assert st["eps"] == st_ref["eps"]


def test_noalloc_allocates_nothing_and_only_enqueues(L):
    """After the set-up-only call, a run leaves the device's free memory as it
    was; with no stats requested the call returns before the run finishes."""
    pr, cfg, seed = CASES[0]
    ref, _ = _context_api(L, pr, seed, cfg)
    x0, prec = _inputs(pr)
    outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
    L.noalloc_setup()
    L.run_noalloc(pr.kind, pr.d, pr.M, x0, seed, outs[0], prec=prec, banana_sb=pr.banana_sb, **cfg)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    L.run_noalloc(pr.kind, pr.d, pr.M, x0, seed, outs[1], prec=prec, banana_sb=pr.banana_sb,
                  stats=False, **cfg)
    pending = not stream.query()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert pending  # a 400-step run of 1000 chains takes milliseconds
    assert torch.equal(outs[0], ref) and torch.equal(outs[1], ref)


def test_noalloc_rejects_what_it_does_not_serve(L):
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LapsError) as err:
        # 200000 steps: the moving window alone (T = 40000 rows of d = 100) needs 32 MB
        L.run_noalloc(L.BANANA, 100, 256, None, 0, out, n_total_steps=200000)
    assert err.value.status == 1 and "bytes of scratch" in str(err.value)
    for kw in ({"precision": 1}, {"stop_b2": 0.01}, {"dtilde_K": 4}):
        with pytest.raises(L.LapsError) as err:
            L.run_noalloc(L.BANANA, 20, 64, None, 0, out, n_total_steps=100, **kw)
        assert err.value.status == 6, kw  # LAPS_ERR_UNSUPPORTED
