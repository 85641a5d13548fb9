"""The oracle's Philox4x32-10 against cuRAND's.

Every parity test feeds the oracle and the CUDA library the same Philox
stream, and both restate the generator of Salmon, Moraes, Dror and Shaw
(SC'11) from its definition; a shared misreading (a wrong multiplier, Weyl
constant or word order) would pass every test that compares the two.  Here
the oracle's generator is compared bit for bit with the round function of
cuRAND's device header (curand_Philox4x32_10), an implementation this
repository did not write, on 2^20 random (counter, key) pairs and on the
counter/key corners.  The probe kernel (tests/gpu_src/curand_philox.cu) is
compiled by this test with nvcc.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gpu_src", "curand_philox.cu")


@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16696_gb300 import build
    so = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    cmd = [build._nvcc(), *build.ARCH, "-O2", "-shared", "-Xcompiler", "-fPIC", SRC, "-o", so]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lib = C.CDLL(so)
    lib.curand_philox_ref.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    lib.curand_philox_ref.restype = C.c_int

    def run(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
        n = ctr.shape[0]
        c = torch.from_numpy(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).cuda()
        k = torch.from_numpy(np.ascontiguousarray(key, dtype=np.uint32).view(np.int32)).cuda()
        o = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        st = lib.curand_philox_ref(c.data_ptr(), k.data_ptr(), o.data_ptr(), n,
                                   torch.cuda.current_stream().cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        return o.cpu().numpy().view(np.uint32)

    return run


def _oracle_by_key(ora, ctr, key):
    """The oracle's Philox row by row, grouped by key (its batch call takes one key)."""
    out = np.empty_like(ctr)
    keys, inv = np.unique(key, axis=0, return_inverse=True)
    for j, k in enumerate(keys):
        rows = np.nonzero(inv.ravel() == j)[0]
        out[rows] = ora.philox(ctr[rows], (int(k[0]), int(k[1])))
    return out


def test_oracle_philox_equals_curand_random_pairs(curand_philox, ora):
    rng = np.random.default_rng(20260116)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    # 64 random keys, so that the oracle's one-key batch call serves 2^14 rows each
    keys = rng.integers(0, 2**32, size=(64, 2), dtype=np.uint64).astype(np.uint32)
    key = keys[rng.integers(0, 64, size=n)]
    np.testing.assert_array_equal(_oracle_by_key(ora, ctr, key), curand_philox(ctr, key))


def test_oracle_philox_equals_curand_corners(curand_philox, ora):
    """All-zero and all-one words, single bits, and the counters the sampler
    uses (coordinate block, chain, step, tag | pid << 8) under the seeds the
    tests use."""
    ctr, key = [], []
    words = [0, 1, 0x80000000, 0xFFFFFFFF, 0x12345678]
    for w0 in words:
        for w in range(4):
            c = [0, 0, 0, 0]
            c[w] = w0
            for k in ((0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (1, 0), (0, 1)):
                ctr.append(c)
                key.append(k)
    for seed in (0, 3, 7, 0x0123456789ABCDEF):
        for (j, m, t, tag, pid) in ((0, 0, 0, 0, 0), (24, 4095, 4999, 2, 0), (2499, 16383, 1999, 1, 64),
                                    (0, 255, 0xFFFFFFFF, 1, 0), (0, 8191, 132, 4, 0)):
            ctr.append([j, m, t, tag | (pid << 8)])
            key.append([seed & 0xFFFFFFFF, seed >> 32])
    ctr = np.array(ctr, dtype=np.uint64).astype(np.uint32)
    key = np.array(key, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(_oracle_by_key(ora, ctr, key), curand_philox(ctr, key))
