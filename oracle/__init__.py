"""FP64 CPU oracle of LAPS -- TEST INFRASTRUCTURE ONLY.

Loaded by ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``; nothing in the product package imports
it.  The C source (``laps_oracle.c``) is a plain restatement of Algorithm 1 and
Apps. E-F of the paper; this module only compiles it with gcc on first use and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "laps_oracle.c")
_HDR = os.path.join(_HERE, "laps_oracle.h")
_SO = os.path.join(_HERE, "liblaps_oracle.so")
_lock = threading.Lock()
_lib = None

GAUSS_DIAG, BANANA, FUNNEL, LOGREG, GAUSS_DENSE = 0, 1, 2, 3, 4
LF, MN2, MN4 = 0, 1, 2
TAG_X0, TAG_O1, TAG_O2, TAG_REFRESH, TAG_MH = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C11, OpenMP, -lm)."""
    stale = (not os.path.exists(_SO)) or any(
        os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _SO)
    return _SO


class Target(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int64), ("prec", C.POINTER(C.c_double)),
                ("banana_sb", C.c_double), ("funnel_sv", C.c_double), ("n_data", C.c_int64),
                ("X", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("prior_var", C.c_double)]


class Config(C.Structure):
    _fields_ = [("C", C.c_double), ("alpha", C.c_double), ("switch_tol", C.c_double),
                ("window_frac", C.c_double), ("acc_tol", C.c_double),
                ("adj_L_factor", C.c_double), ("eps0_coef", C.c_double),
                ("a_target_mn2", C.c_double), ("a_target_mn4", C.c_double),
                ("n_total_steps", C.c_int), ("steps_per_proposal", C.c_int),
                ("mn4_min_dim", C.c_int), ("eevpd_centered", C.c_int), ("adjusted", C.c_int),
                ("force_switch_at", C.c_int), ("fixed_eps", C.c_double),
                ("round_state_f32", C.c_int), ("dtilde_K", C.c_int)]


class TraceRow(C.Structure):
    _fields_ = [("phase", C.c_int), ("t", C.c_int), ("eps", C.c_double), ("L", C.c_double),
                ("eps_used", C.c_double), ("eevpd", C.c_double), ("eevpd_wanted", C.c_double),
                ("dtilde", C.c_double), ("max_delta", C.c_double), ("acc", C.c_double),
                ("b2_max", C.c_double), ("b2_avg", C.c_double), ("sum_var", C.c_double),
                ("nonfinite", C.c_int), ("adapting", C.c_int), ("grads", C.c_longlong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.ora_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.ora_uniform.argtypes = [C.c_uint32]
            L.ora_uniform.restype = C.c_double
            L.ora_philox_batch.argtypes = [C.c_int64, _u32p, _u32p, _u32p]
            L.ora_normals_chains.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32,
                                             C.c_uint32, C.c_uint32, C.c_int64, _dp]
            L.ora_logp_grad.argtypes = [C.POINTER(Target), _dp, _dp]
            L.ora_logp_grad.restype = C.c_double
            L.ora_logp_grad_batch.argtypes = [C.POINTER(Target), C.c_int64, _dp, _dp, _dp]
            L.ora_O.argtypes = [C.c_int64, C.c_double, C.c_double, _dp, _dp]
            L.ora_A.argtypes = [C.c_int64, C.c_double, _dp, _dp]
            L.ora_B.argtypes = [C.c_int64, C.c_double, _dp, _dp]
            L.ora_B.restype = C.c_double
            L.ora_integrator_coefs.argtypes = [C.c_int, _dp, _dp]
            L.ora_integrator_coefs.restype = C.c_int
            L.ora_Phi.argtypes = [C.POINTER(Target), C.c_int, C.c_double, _dp, _dp, _dp, _dp]
            L.ora_Phi.restype = C.c_double
            L.ora_F.argtypes = [C.c_double]
            L.ora_F.restype = C.c_double
            L.ora_dtilde_diag.argtypes = [C.c_int64, C.c_int64, _dp, _dp]
            L.ora_dtilde_diag.restype = C.c_double
            L.ora_dtilde_full.argtypes = [C.c_int64, C.c_int64, _dp, _dp, C.c_int, C.c_uint64,
                                          C.c_uint32, C.c_uint32]
            L.ora_dtilde_full.restype = C.c_double
            L.ora_rademacher.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                         C.c_int64]
            L.ora_rademacher.restype = C.c_double
            L.ora_L_of.argtypes = [C.c_int64, C.c_int64, _dp, C.c_double]
            L.ora_L_of.restype = C.c_double
            L.ora_rel_fluct.argtypes = [C.c_int64, _dp]
            L.ora_rel_fluct.restype = C.c_double
            L.ora_bisect.argtypes = [C.c_double, C.c_double, C.c_double, _dp, _dp]
            L.ora_bisect.restype = C.c_double
            L.ora_config_default.argtypes = [C.POINTER(Config)]
            L.ora_create.argtypes = [C.POINTER(Target), C.POINTER(Config), C.c_int64, _dp,
                                     C.c_uint64, C.c_uint32]
            L.ora_create.restype = C.c_void_p
            L.ora_destroy.argtypes = [C.c_void_p]
            L.ora_set_truth.argtypes = [C.c_void_p, _dp, _dp]
            L.ora_row0.argtypes = [C.c_void_p, C.POINTER(TraceRow)]
            L.ora_iterate.argtypes = [C.c_void_p, C.POINTER(TraceRow)]
            L.ora_iterate.restype = C.c_int
            L.ora_get_x.argtypes = [C.c_void_p, _dp]
            L.ora_get_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            L.ora_get_sigma.argtypes = [C.c_void_p, _dp]
            for fn in ("ora_phase", "ora_t", "ora_t_switch", "ora_window_T", "ora_integrator"):
                getattr(L, fn).argtypes = [C.c_void_p]
                getattr(L, fn).restype = C.c_int
            L.ora_mams_proposal.argtypes = [C.POINTER(Target), C.c_int, C.c_double, C.c_double,
                                            C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                            C.c_uint32, C.c_uint32, _dp, _dp, _dp, _dp,
                                            C.POINTER(C.c_int), _dp]
            L.ora_mams_proposal.restype = C.c_double
            L.ora_mams_batch.argtypes = [C.POINTER(Target), C.c_int, C.c_double, C.c_double,
                                         C.c_int, C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32,
                                         C.c_uint32, C.c_int, _dp, _dp, C.POINTER(C.c_int)]
            L.ora_set_threads.argtypes = [C.c_int]
            L.ora_set_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- random stream
def philox(ctrs: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each row of ``ctrs`` ([n, 4] uint32) under ``key`` (2 words)."""
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(ctrs)
    lib().ora_philox_batch(ctrs.shape[0], ctrs.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                           out.ctypes.data_as(_u32p))
    return out


def uniform(r: int) -> float:
    return lib().ora_uniform(int(r))


def normals(seed: int, m0: int, nm: int, t: int, tag: int, pid: int, d: int) -> np.ndarray:
    """[nm, d] standard normals of chains m0..m0+nm-1 under (t, tag, pid)."""
    z = np.empty((nm, d), dtype=np.float64)
    lib().ora_normals_chains(seed, m0, nm, t & 0xFFFFFFFF, tag, pid, d, _p(z))
    return z


# ---------------------------------------------------------------- targets
class OracleTarget:
    """Keeps the numpy buffers a ``Target`` struct points into alive."""

    def __init__(self, kind: int, d: int, prec=None, banana_sb=0.1, funnel_sv=3.0, X=None,
                 y=None, prior_var=1.0):
        self.kind, self.d = kind, d
        self._prec = _f64(prec) if prec is not None else None
        self._X = _f64(X) if X is not None else None
        self._y = _f64(y) if y is not None else None
        n_data = 0 if X is None else self._X.shape[0]
        self.s = Target(kind, d, _p(self._prec) if self._prec is not None else None,
                        banana_sb, funnel_sv, n_data,
                        _p(self._X) if self._X is not None else None,
                        _p(self._y) if self._y is not None else None, prior_var)

    def logp_grad(self, x: np.ndarray):
        """log p and its gradient for one point ([d]) or a batch ([M, d])."""
        x = _f64(x)
        if x.ndim == 1:
            g = np.empty_like(x)
            lp = lib().ora_logp_grad(C.byref(self.s), _p(x), _p(g))
            return lp, g
        g = np.empty_like(x)
        lp = np.empty(x.shape[0], dtype=np.float64)
        lib().ora_logp_grad_batch(C.byref(self.s), x.shape[0], _p(x), _p(lp), _p(g))
        return lp, g


# ---------------------------------------------------------------- maps
def O(eps: float, L: float, z: np.ndarray, u: np.ndarray) -> None:
    lib().ora_O(u.shape[0], eps, L, _p(z), _p(u))


def A(eps: float, u: np.ndarray, x: np.ndarray) -> None:
    lib().ora_A(x.shape[0], eps, _p(u), _p(x))


def B(eps: float, g: np.ndarray, u: np.ndarray) -> float:
    return lib().ora_B(u.shape[0], eps, _p(g), _p(u))


def coefs(integ: int):
    b = np.zeros(8)
    a = np.zeros(8)
    K = lib().ora_integrator_coefs(integ, _p(b), _p(a))
    return b[:K].copy(), a[:K - 1].copy()


def Phi(target: OracleTarget, integ: int, eps: float, x, u, g, logp: float):
    """Deterministic step in place on (x, u, g); returns (energy error, new logp)."""
    lp = C.c_double(logp)
    dl = lib().ora_Phi(C.byref(target.s), integ, eps, _p(x), _p(u), _p(g), C.byref(lp))
    return dl, lp.value


def F(D: float) -> float:
    return lib().ora_F(D)


def dtilde_diag(X: np.ndarray, G: np.ndarray) -> float:
    X, G = _f64(X), _f64(G)
    return lib().ora_dtilde_diag(X.shape[0], X.shape[1], _p(X), _p(G))


def dtilde_full(X: np.ndarray, G: np.ndarray, K: int, seed: int = 0, pid: int = 0,
                t: int = 0) -> float:
    X, G = _f64(X), _f64(G)
    return lib().ora_dtilde_full(X.shape[0], X.shape[1], _p(X), _p(G), K, seed, pid, t)


def rademacher(seed: int, pid: int, t: int, k: int, d: int) -> np.ndarray:
    return np.array([lib().ora_rademacher(seed, pid, t, k, i) for i in range(d)])


def L_of(X: np.ndarray, alpha: float = 2.0) -> float:
    X = _f64(X)
    return lib().ora_L_of(X.shape[0], X.shape[1], _p(X), alpha)


def rel_fluct(hist) -> float:
    h = _f64(hist)
    return lib().ora_rel_fluct(h.shape[0], _p(h))


def bisect(eps: float, a: float, a_target: float, lo: float, hi: float):
    clo, chi = C.c_double(lo), C.c_double(hi)
    e = lib().ora_bisect(eps, a, a_target, C.byref(clo), C.byref(chi))
    return e, clo.value, chi.value


def mams_proposal(target: OracleTarget, integ: int, eps: float, L: float, n_steps: int,
                  seed: int, pid: int, m: int, t0: int, p: int, x, g, logp: float):
    """One MAMS proposal for one chain (no preconditioner); x, g updated in place."""
    u = np.zeros_like(x)
    lp = C.c_double(logp)
    acc = C.c_int(0)
    dl = C.c_double(0)
    a = lib().ora_mams_proposal(C.byref(target.s), integ, eps, L, n_steps, seed, pid, m, t0, p,
                                _p(x), _p(g), C.byref(lp), _p(u), C.byref(acc), C.byref(dl))
    return a, bool(acc.value), dl.value, lp.value


def mams_batch(target: OracleTarget, integ: int, eps: float, L: float, n_steps: int,
               seed: int, X: np.ndarray, pid: int = 0, t0: int = 0, p: int = 0,
               mh_mode: int = 0):
    """One MAMS proposal for every row of X (updated in place).  mh_mode 1 and 2
    plant a mistake (accept all / flipped energy sign) for power checks."""
    assert X.dtype == np.float64 and X.flags.c_contiguous
    M = X.shape[0]
    acc_p = np.empty(M)
    acc = np.empty(M, dtype=np.int32)
    lib().ora_mams_batch(C.byref(target.s), integ, eps, L, n_steps, seed, pid, M, t0, p,
                         mh_mode, _p(X), _p(acc_p), acc.ctypes.data_as(C.POINTER(C.c_int)))
    return acc_p, acc.astype(bool)


def set_threads(n: int) -> int:
    return lib().ora_set_threads(n)


def default_config(**kw) -> Config:
    c = Config()
    lib().ora_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


# ---------------------------------------------------------------- full LAPS
class OracleLAPS:
    """Algorithm 1 on an ensemble of M chains (all state FP64 on the host)."""

    def __init__(self, target: OracleTarget, x0: np.ndarray, seed: int, pid: int = 0,
                 config: Config | None = None, truth=None, **cfg_kw):
        self.target = target
        self.cfg = config if config is not None else default_config(**cfg_kw)
        x0 = _f64(x0)
        self.M, self.d = x0.shape
        self._h = lib().ora_create(C.byref(target.s), C.byref(self.cfg), self.M, _p(x0),
                                   seed, pid)
        if truth is not None:
            ex2, vx2 = _f64(truth[0]), _f64(truth[1])
            lib().ora_set_truth(self._h, _p(ex2), _p(vx2))
        r = TraceRow()
        lib().ora_row0(self._h, C.byref(r))
        self.trace = [r.as_dict()]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    def iterate(self, n: int = 1) -> int:
        done = 0
        r = TraceRow()
        for _ in range(n):
            if not lib().ora_iterate(self._h, C.byref(r)):
                break
            self.trace.append(r.as_dict())
            done += 1
        return done

    def run(self) -> int:
        return self.iterate(1 << 30)

    def x(self) -> np.ndarray:
        out = np.empty((self.M, self.d))
        lib().ora_get_x(self._h, _p(out))
        return out

    def state(self):
        y, u, g = (np.empty((self.M, self.d)) for _ in range(3))
        lp = np.empty(self.M)
        lib().ora_get_state(self._h, _p(y), _p(u), _p(g), _p(lp))
        return y, u, g, lp

    def sigma(self) -> np.ndarray:
        s = np.empty(self.d)
        lib().ora_get_sigma(self._h, _p(s))
        return s

    @property
    def phase(self) -> int:
        return lib().ora_phase(self._h)

    @property
    def t(self) -> int:
        return lib().ora_t(self._h)

    @property
    def t_switch(self) -> int:
        return lib().ora_t_switch(self._h)

    @property
    def window_T(self) -> int:
        return lib().ora_window_T(self._h)

    @property
    def integrator(self) -> int:
        return lib().ora_integrator(self._h)
