"""ctypes binding of liblaps.so (include/laps.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and streams, and raises on any non-OK status.
There is no fallback: without the built library (``build.py``) every call
raises ``LapsError``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblaps.so")

GAUSS_DIAG, BANANA, FUNNEL, LOGREG, GAUSS_DENSE, USER = 0, 1, 2, 3, 4, 5
FP32, MIXED, BF16X3, MIXED_BF16X3 = 0, 1, 2, 3
LF, MN2, MN4 = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "NONFINITE",
          6: "UNSUPPORTED"}


class LapsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("LAPS_ERR_%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


# int (*)(const float* x, int64 M, int64 ld, float* logp, float* grad, void* stream, void* user)
LOGP_GRAD_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p)


class TargetDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int64), ("prec", C.c_void_p),
                ("banana_sb", C.c_double), ("funnel_sv", C.c_double), ("n_data", C.c_int64),
                ("X", C.c_void_p), ("y", C.c_void_p), ("prior_var", C.c_double),
                ("user_fn", LOGP_GRAD_FN), ("user_data", C.c_void_p)]


class _DeviceView:
    """A float32 device array given by pointer, shape and byte strides, for
    torch.as_tensor (zero-copy, through __cuda_array_interface__)."""

    def __init__(self, ptr: int, shape, strides):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": "<f4", "strides": tuple(strides), "version": 3}


class Config(C.Structure):
    _fields_ = [("C", C.c_double), ("alpha", C.c_double), ("switch_tol", C.c_double),
                ("window_frac", C.c_double), ("acc_tol", C.c_double),
                ("adj_L_factor", C.c_double), ("eps0_coef", C.c_double),
                ("a_target_mn2", C.c_double), ("a_target_mn4", C.c_double),
                ("n_total_steps", C.c_int), ("steps_per_proposal", C.c_int),
                ("mn4_min_dim", C.c_int), ("eevpd_centered", C.c_int), ("adjusted", C.c_int),
                ("force_switch_at", C.c_int), ("fixed_eps", C.c_double),
                ("stop_b2", C.c_double), ("stop_b2_max", C.c_int),
                ("precision", C.c_int), ("barrier_timeout_ns", C.c_int64),
                ("chains_per_block", C.c_int), ("lanes_per_chain", C.c_int),
                ("coords_per_lane", C.c_int), ("barrier_extra_arrivals", C.c_int),
                ("dtilde_K", C.c_int), ("dense_streamed", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("phase", C.c_int), ("t", C.c_int), ("t_switch", C.c_int),
                ("integrator", C.c_int), ("adapting", C.c_int), ("done", C.c_int),
                ("iterations", C.c_int), ("nonfinite_total", C.c_int), ("grads", C.c_longlong),
                ("eps", C.c_double), ("L", C.c_double), ("eevpd", C.c_double),
                ("eevpd_wanted", C.c_double), ("dtilde", C.c_double), ("max_delta", C.c_double),
                ("acc", C.c_double), ("b2_max", C.c_double), ("b2_avg", C.c_double),
                ("sum_var", C.c_double), ("b2_first_t", C.c_int),
                ("b2_first_grads", C.c_longlong), ("b2_first_ns", C.c_double)]


class TraceRow(C.Structure):
    _fields_ = [("phase", C.c_int), ("t", C.c_int), ("eps", C.c_double), ("L", C.c_double),
                ("eps_used", C.c_double), ("eevpd", C.c_double), ("eevpd_wanted", C.c_double),
                ("dtilde", C.c_double), ("max_delta", C.c_double), ("acc", C.c_double),
                ("b2_max", C.c_double), ("b2_avg", C.c_double), ("sum_var", C.c_double),
                ("nonfinite", C.c_int), ("adapting", C.c_int), ("grads", C.c_longlong),
                ("time_ns", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("d", C.c_int64), ("M", C.c_int64), ("prec", C.c_void_p), ("x0", C.c_void_p),
                ("x0_scale", C.c_double)]


class BatchShape(C.Structure):
    _fields_ = [("coords_per_lane", C.c_int), ("widen", C.c_int), ("slice", C.c_int),
                ("threads", C.c_int), ("blocks", C.c_int), ("tuned", C.c_int)]


class LaunchInfo(C.Structure):
    _fields_ = [("chains_per_block", C.c_int), ("lanes_per_chain", C.c_int),
                ("coords_per_lane", C.c_int), ("threads", C.c_int), ("blocks", C.c_int),
                ("resident", C.c_int)]


class Peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int), ("sm_mhz", C.c_double), ("fp32_tflops", C.c_double),
                ("fp64_tflops", C.c_double), ("ex2_per_clk_sm", C.c_double),
                ("grid_barrier_us", C.c_double), ("barrier_blocks", C.c_int)]


def _as_dict(s):
    return {n: getattr(s, n) for n, _ in s._fields_}


_lock = threading.Lock()
_lib = None
_vp = C.c_void_p

# name -> (restype, argtypes); the list is also the ABI the tests check
SIGNATURES = {
    "laps_config_default": (None, [C.POINTER(Config)]),
    "laps_last_error": (C.c_char_p, []),
    "laps_version": (C.c_char_p, []),
    "laps_target_create": (C.c_int, [C.POINTER(TargetDesc), C.POINTER(_vp)]),
    "laps_target_destroy": (None, [_vp]),
    "laps_target_logp_grad": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "laps_target_logp_grad_prec": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, C.c_int, _vp]),
    "laps_target_status": (C.c_int, [_vp]),
    "laps_create": (C.c_int, [_vp, C.c_int64, C.POINTER(Config), C.POINTER(_vp)]),
    "laps_create_sharded": (C.c_int, [_vp, C.c_int64, C.c_void_p, C.POINTER(Config), C.POINTER(_vp)]),
    "laps_destroy": (None, [_vp]),
    "laps_init": (C.c_int, [_vp, _vp, C.c_double, C.c_uint64, _vp]),
    "laps_step": (C.c_int, [_vp, C.c_int, _vp]),
    "laps_run": (C.c_int, [_vp, _vp]),
    "laps_adapt_freeze": (C.c_int, [_vp, C.c_int]),
    "laps_sample": (C.c_int, [_vp, _vp, _vp]),
    "laps_get_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "laps_set_truth": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "laps_get_stats": (C.c_int, [_vp, C.POINTER(Stats)]),
    "laps_get_trace": (C.c_int, [_vp, C.POINTER(TraceRow), C.c_int, C.POINTER(C.c_int)]),
    "laps_checkpoint": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "laps_restore": (C.c_int, [_vp, _vp, C.c_size_t]),
    "laps_philox": (C.c_int, [_vp, C.c_uint64, _vp, C.c_int64, _vp]),
    "laps_normals": (C.c_int, [C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32, C.c_uint32,
                               C.c_uint32, C.c_int64, _vp, _vp]),
    "laps_get_launch_info": (C.c_int, [_vp, C.POINTER(LaunchInfo)]),
    "laps_measure_peaks": (C.c_int, [C.POINTER(Peaks), _vp]),
    "laps_run_noalloc": (C.c_int, [C.POINTER(TargetDesc), C.c_int64, C.POINTER(Config), _vp,
                                   C.c_double, C.c_uint64, _vp, C.POINTER(Stats), _vp]),
    "laps_batch_create": (C.c_int, [C.POINTER(Problem), C.c_int, C.POINTER(Config),
                                    C.POINTER(_vp)]),
    "laps_batch_destroy": (None, [_vp]),
    "laps_batch_set_truth": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    "laps_batch_init": (C.c_int, [_vp, C.c_uint64, _vp]),
    "laps_batch_step": (C.c_int, [_vp, C.c_int, _vp]),
    "laps_batch_run": (C.c_int, [_vp, C.c_int, _vp]),
    "laps_batch_tune": (C.c_int, [_vp, _vp]),
    "laps_batch_get_shape": (C.c_int, [_vp, C.POINTER(BatchShape)]),
    "laps_batch_set_shape": (C.c_int, [_vp, C.POINTER(BatchShape)]),
    "laps_batch_get_stats": (C.c_int, [_vp, C.c_int, C.POINTER(Stats)]),
    "laps_batch_get_trace": (C.c_int, [_vp, C.c_int, C.POINTER(TraceRow), C.c_int,
                                       C.POINTER(C.c_int)]),
    "laps_batch_sample": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "laps_batch_partition": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int, C.c_int,
                                       C.POINTER(C.c_int32)]),
    "laps_batch_set_ids": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
}


def lib(path: str | None = None):
    """Load liblaps.so (raises LapsError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise LapsError(2, "liblaps.so not built (%s); run paper_2601_16696_gb300/build.py"
                                % p)
            L = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise LapsError(st, lib().laps_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t: torch.Tensor | None, dtype=torch.float32):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor of %s" % dtype)
    return C.c_void_p(t.data_ptr())


def default_config(**kw) -> Config:
    c = Config()
    lib().laps_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class Target:
    """A built-in target (device copies of its parameters are kept alive here)."""

    def __init__(self, kind: int, d: int, prec=None, banana_sb: float = 0.1,
                 funnel_sv: float = 3.0, X=None, y=None, prior_var: float = 1.0,
                 device="cuda"):
        self.kind, self.d = kind, d
        self._keep = []
        desc = TargetDesc(kind, d, None, banana_sb, funnel_sv, 0, None, None, prior_var)
        if prec is not None:
            p = torch.as_tensor(prec, dtype=torch.float32, device=device).contiguous()
            self._keep.append(p)
            desc.prec = p.data_ptr()
        if X is not None:
            Xt = torch.as_tensor(X, dtype=torch.float32, device=device).contiguous()
            yt = torch.as_tensor(y, dtype=torch.float32, device=device).contiguous()
            self._keep += [Xt, yt]
            desc.X, desc.y, desc.n_data = Xt.data_ptr(), yt.data_ptr(), Xt.shape[0]
        h = C.c_void_p()
        _check(lib().laps_target_create(C.byref(desc), C.byref(h)))
        self._h = h

    @classmethod
    def from_callable(cls, d: int, fn):
        """A LAPS_USER target: fn(x, logp, grad) receives torch views of the
        ensemble's points x [M, d] and fills logp [M] and grad [M, d] (grad log p)
        with torch operations.  It runs on the sampler's stream, once per
        gradient evaluation; an exception in fn makes the sampler call raise."""
        self = cls.__new__(cls)
        self.kind, self.d, self._keep, self._errors = USER, d, [], []

        def cb(x, M, ld, lp, g, stream, user):
            try:
                if M == 0:
                    return 0
                xv = torch.as_tensor(_DeviceView(x, (M, ld), (4 * ld, 4)), device="cuda")[:, :d]
                gv = torch.as_tensor(_DeviceView(g, (M, ld), (4 * ld, 4)), device="cuda")[:, :d]
                lv = torch.as_tensor(_DeviceView(lp, (M,), (4,)), device="cuda")
                st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(st):
                    fn(xv, lv, gv)
                return 0
            except Exception as e:  # reported by the laps call that made this one
                self._errors.append(e)
                return 1

        cfn = LOGP_GRAD_FN(cb)
        self._keep.append(cfn)
        desc = TargetDesc(USER, d, None, 0.1, 3.0, 0, None, None, 1.0, cfn, None)
        h = C.c_void_p()
        _check(lib().laps_target_create(C.byref(desc), C.byref(h)))
        self._h = h
        return self

    @classmethod
    def from_problem(cls, pr, device="cuda"):
        return cls(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb, funnel_sv=pr.funnel_sv,
                   X=pr.X, y=pr.y, prior_var=pr.prior_var, device=device)

    @property
    def handle(self):
        return self._h

    def logp_grad(self, x: torch.Tensor, precision: int = 0, stream=None):
        """log p [M] and grad log p [M, d] of the rows of x (FP32, CUDA);
        precision 1 (LAPS_MIXED): the BF16 tensor-core form of a LOGREG target;
        2 (LAPS_BF16X3): its tensor-core form at FP32 accuracy."""
        x = x.contiguous()
        M = x.shape[0]
        logp = torch.empty(M, dtype=torch.float32, device=x.device)
        grad = torch.empty_like(x)
        if precision == 0:
            _check(lib().laps_target_logp_grad(self._h, _ptr(x), M, _ptr(logp), _ptr(grad),
                                               _stream(stream)))
        else:
            _check(lib().laps_target_logp_grad_prec(self._h, _ptr(x), M, _ptr(logp), _ptr(grad),
                                                    precision, _stream(stream)))
        return logp, grad

    def check(self):
        """Raises LapsError if a kernel of this target latched an error."""
        _check(lib().laps_target_status(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.laps_target_destroy(h)
            self._h = None


_ALLGATHER = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class ShardSpec(C.Structure):
    _fields_ = [("M_total", C.c_int64), ("m0", C.c_int64), ("rank", C.c_int), ("n_ranks", C.c_int),
                ("allgather", _ALLGATHER), ("user_data", C.c_void_p)]


class _DeviceBytes:
    """A device range seen by torch (no copy) through the CUDA array interface."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_bytes(ptr: int, nbytes: int) -> torch.Tensor:
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")


def nccl_allgather(group=None):
    """The exchange of a chain-sharded ensemble over torch.distributed (NCCL):
    gathers every rank's totals in rank order on the sampler's stream."""
    import torch.distributed as dist

    def gather(send: int, recv: int, nbytes: int, stream: int):
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            dist.all_gather_into_tensor(device_bytes(recv, nbytes * dist.get_world_size(group)),
                                        device_bytes(send, nbytes), group=group)
    return gather


class Sampler:
    """One LAPS run of M chains on a Target (Algorithm 1 on the GPU).

    shard: None, or (M_total, m0, rank, n_ranks, allgather) for a chain-sharded
    ensemble (laps_create_sharded): this sampler holds chains m0 .. m0 + M - 1 of
    M_total; allgather(send_ptr, recv_ptr, nbytes, stream_ptr) gathers every
    rank's totals (device memory) in rank order on that stream, e.g.
    nccl_allgather(); None with one rank."""

    def __init__(self, target: Target, M: int, config: Config | None = None, shard=None, **cfg_kw):
        self.target, self.M, self.d = target, M, target.d
        self.config = config if config is not None else default_config(**cfg_kw)
        h = C.c_void_p()
        if shard is None:
            _check(lib().laps_create(target.handle, M, C.byref(self.config), C.byref(h)))
        else:
            M_total, m0, rank, n_ranks, fn = shard

            def cb(send, recv, nbytes, stream, user):
                try:
                    fn(send, recv, nbytes, stream)
                    return 0
                except Exception:  # reported by the library as a failed callback
                    import traceback
                    traceback.print_exc()
                    return 1
            self._cb = _ALLGATHER(cb) if fn is not None else _ALLGATHER()
            spec = ShardSpec(M_total, m0, rank, n_ranks, self._cb, None)
            self._spec = spec
            _check(lib().laps_create_sharded(target.handle, M, C.cast(C.pointer(spec), C.c_void_p),
                                             C.byref(self.config), C.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.laps_destroy(h)
            self._h = None

    def set_truth(self, Ex2, Varx2):
        a = (C.c_double * self.d)(*[float(v) for v in Ex2])
        b = (C.c_double * self.d)(*[float(v) for v in Varx2])
        _check(lib().laps_set_truth(self._h, a, b))

    def init(self, x0: torch.Tensor | None = None, x0_scale: float = 1.0, seed: int = 0,
             stream=None):
        self._x0 = x0.contiguous() if x0 is not None else None
        _check(lib().laps_init(self._h, _ptr(self._x0), x0_scale, seed, _stream(stream)))

    def step(self, n: int = 1, stream=None):
        _check(lib().laps_step(self._h, n, _stream(stream)))

    def run(self, stream=None):
        _check(lib().laps_run(self._h, _stream(stream)))

    def freeze(self, frozen: bool = True):
        _check(lib().laps_adapt_freeze(self._h, int(frozen)))

    def sample(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.M, self.d, dtype=torch.float32, device="cuda")
        _check(lib().laps_sample(self._h, _ptr(out), _stream(stream)))
        return out

    def state(self, stream=None):
        y, u, g = (torch.empty(self.M, self.d, dtype=torch.float32, device="cuda")
                   for _ in range(3))
        lp = torch.empty(self.M, dtype=torch.float64, device="cuda")
        sg = torch.empty(self.d, dtype=torch.float32, device="cuda")
        _check(lib().laps_get_state(self._h, _ptr(y), _ptr(u), _ptr(g),
                                    _ptr(lp, torch.float64), _ptr(sg), _stream(stream)))
        return y, u, g, lp, sg

    def stats(self) -> dict:
        s = Stats()
        _check(lib().laps_get_stats(self._h, C.byref(s)))
        return _as_dict(s)

    def stats_status(self):
        """(status code, stats dict) without raising."""
        s = Stats()
        st = lib().laps_get_stats(self._h, C.byref(s))
        return st, _as_dict(s)

    def trace(self) -> list:
        n = C.c_int(0)
        _check(lib().laps_get_trace(self._h, None, 0, C.byref(n)))
        rows = (TraceRow * max(1, n.value))()
        _check(lib().laps_get_trace(self._h, rows, n.value, C.byref(n)))
        return [_as_dict(rows[i]) for i in range(n.value)]

    def checkpoint(self) -> bytes:
        sz = C.c_size_t(0)
        _check(lib().laps_checkpoint(self._h, None, C.byref(sz)))
        buf = C.create_string_buffer(sz.value)
        _check(lib().laps_checkpoint(self._h, buf, C.byref(sz)))
        return buf.raw[:sz.value]

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().laps_restore(self._h, buf, len(blob)))

    def launch_info(self) -> dict:
        li = LaunchInfo()
        _check(lib().laps_get_launch_info(self._h, C.byref(li)))
        return _as_dict(li)


def measure_peaks(stream=None) -> dict:
    """Throughput probes of the current GPU (FP32 / FP64 FMA, ex2 per clock,
    grid-barrier latency, SM clock); synchronises the stream."""
    p = Peaks()
    _check(lib().laps_measure_peaks(C.byref(p), _stream(stream)))
    return _as_dict(p)


def philox(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Philox4x32-10 of int32 counters ctr [n, 4] (CUDA), as the sampler draws it."""
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check(lib().laps_philox(_ptr(ctr, torch.int32), seed, _ptr(out, torch.int32), ctr.shape[0],
                             _stream(stream)))
    return out


def normals(seed: int, m0: int, nm: int, t: int, tag: int, pid: int, d: int,
            stream=None) -> torch.Tensor:
    out = torch.empty(nm, d, dtype=torch.float32, device="cuda")
    _check(lib().laps_normals(seed, m0, nm, t & 0xFFFFFFFF, tag, pid, d, _ptr(out),
                              _stream(stream)))
    return out


def run_noalloc(kind: int, d: int, M: int, x0: torch.Tensor | None, seed: int,
                out: torch.Tensor, prec: torch.Tensor | None = None, banana_sb: float = 0.1,
                funnel_sv: float = 3.0, x0_scale: float = 1.0, config: Config | None = None,
                stream=None, stats: bool = True, **cfg_kw) -> dict | None:
    """One whole LAPS run through laps_run_noalloc (no device allocation in the
    library); samples are written to ``out`` [M, d].  Returns the final stats
    (the call then synchronises the stream), or None with ``stats=False`` (the
    call only enqueues the run)."""
    cfg = config if config is not None else default_config(**cfg_kw)
    desc = TargetDesc(kind, d, prec.data_ptr() if prec is not None else None, banana_sb,
                      funnel_sv, 0, None, None, 1.0)
    s = Stats()
    _check(lib().laps_run_noalloc(C.byref(desc), M, C.byref(cfg), _ptr(x0), x0_scale, seed,
                                  _ptr(out), C.byref(s) if stats else None, _stream(stream)))
    return _as_dict(s) if stats else None


def noalloc_setup() -> None:
    """The set-up-only call of laps_run_noalloc: loads its scratch array on the
    current device and looks up its address, nothing else."""
    _check(lib().laps_run_noalloc(None, 0, None, None, 0.0, 0, None, None, None))


def partition_problems(problems, n_ranks: int) -> list:
    """laps_batch_partition: the problem indices each of n_ranks ranks runs
    (``problems``: objects with d and M)."""
    n = len(problems)
    d = np.array([int(p.d) for p in problems], dtype=np.int64)
    M = np.array([int(p.M) for p in problems], dtype=np.int64)
    owner = np.zeros(n, dtype=np.int32)
    _check(lib().laps_batch_partition(d.ctypes.data_as(C.POINTER(C.c_int64)),
                                      M.ctypes.data_as(C.POINTER(C.c_int64)), n, n_ranks,
                                      owner.ctypes.data_as(C.POINTER(C.c_int32))))
    return [[k for k in range(n) if owner[k] == r] for r in range(n_ranks)]


class Batch:
    """Independent diagonal-Gaussian problems in one persistent launch
    (laps_batch_*).  ``problems``: objects with d, M, prec (and optionally x0);
    ``ids``: their Philox problem ids (default 0 .. n-1; a rank's share of a
    partitioned batch passes the problems' indices in the whole batch)."""

    def __init__(self, problems, config: Config | None = None, x0_scale: float = 1.0,
                 use_x0: bool = True, ids=None, **cfg_kw):
        self.config = config if config is not None else default_config(**cfg_kw)
        self.n = len(problems)
        self.dims = [(int(p.d), int(p.M)) for p in problems]
        self._keep = []
        arr = (Problem * self.n)()
        for k, p in enumerate(problems):
            pr = torch.as_tensor(p.prec, dtype=torch.float32, device="cuda").contiguous()
            self._keep.append(pr)
            x0 = None
            if use_x0 and getattr(p, "x0", None) is not None:
                x0 = torch.as_tensor(p.x0, dtype=torch.float32, device="cuda").contiguous()
                self._keep.append(x0)
            arr[k] = Problem(p.d, p.M, pr.data_ptr(), x0.data_ptr() if x0 is not None else None,
                             x0_scale)
        h = C.c_void_p()
        _check(lib().laps_batch_create(arr, self.n, C.byref(self.config), C.byref(h)))
        self._h = h
        if ids is not None:
            a = np.ascontiguousarray(ids, dtype=np.int32)
            if a.shape != (self.n,):
                raise ValueError("ids must hold one id per problem")
            _check(lib().laps_batch_set_ids(self._h, a.ctypes.data_as(C.POINTER(C.c_int32))))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.laps_batch_destroy(h)
            self._h = None

    def set_truth(self, k: int, Ex2, Varx2):
        a = np.ascontiguousarray(Ex2, dtype=np.float64)
        b = np.ascontiguousarray(Varx2, dtype=np.float64)
        _check(lib().laps_batch_set_truth(self._h, k, a.ctypes.data_as(C.POINTER(C.c_double)),
                                          b.ctypes.data_as(C.POINTER(C.c_double))))

    def init(self, seed: int = 0, stream=None):
        _check(lib().laps_batch_init(self._h, seed, _stream(stream)))

    def step(self, n: int = 1, stream=None):
        _check(lib().laps_batch_step(self._h, n, _stream(stream)))

    def run(self, iters_per_launch: int = 64, stream=None):
        _check(lib().laps_batch_run(self._h, iters_per_launch, _stream(stream)))

    def tune(self, stream=None):
        _check(lib().laps_batch_tune(self._h, _stream(stream)))

    def shape(self) -> dict:
        s = BatchShape()
        _check(lib().laps_batch_get_shape(self._h, C.byref(s)))
        return _as_dict(s)

    def set_shape(self, coords_per_lane: int, widen: int = 0, slice: int = 64):
        s = BatchShape(coords_per_lane, widen, slice, 0, 0, 0)
        _check(lib().laps_batch_set_shape(self._h, C.byref(s)))

    def stats(self, k: int) -> dict:
        s = Stats()
        _check(lib().laps_batch_get_stats(self._h, k, C.byref(s)))
        return _as_dict(s)

    def trace(self, k: int) -> list:
        n = C.c_int(0)
        _check(lib().laps_batch_get_trace(self._h, k, None, 0, C.byref(n)))
        rows = (TraceRow * max(1, n.value))()
        _check(lib().laps_batch_get_trace(self._h, k, rows, n.value, C.byref(n)))
        return [_as_dict(rows[i]) for i in range(n.value)]

    def sample(self, k: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        d, M = self.dims[k]
        if out is None:
            out = torch.empty(M, d, dtype=torch.float32, device="cuda")
        elif out.numel() != M * d:
            raise ValueError("out must hold %d x %d values" % (M, d))
        _check(lib().laps_batch_sample(self._h, k, _ptr(out), _stream(stream)))
        return out
