"""LAPS (Late Adjusted Parallel Sampler) ensemble step for GB300 (sm_103a).

The sampler runs in the CUDA library ``liblaps.so`` (built from ``csrc/`` by
``build.py``); :mod:`.laps` is a thin ctypes binding over its C ABI
(``include/laps.h``).  Importing this package does not load the library;
the first call into :mod:`.laps` does, and fails loudly if it is missing.
"""
__all__ = ["laps", "workloads"]
