"""B300-native (sm_103a) batched Relay-BP decoding of ZSZ-LP detector error models.

The compute path lives in ``librelaybp.so`` (CUDA, C ABI in include/relaybp.h);
``paper_2607_27644_b300.relaybp`` is its thin binding (importing it fails
loudly if the library has not been built) and ``stats`` holds the host-side
statistics (Clopper-Pearson intervals, per-round logical error rates).
``build`` compiles the library and is importable without it.
"""
__all__ = ["relaybp", "stats", "build"]
