"""GB300-native bulk AES (ECB, plus CTR and CBC decryption) behind a C ABI.

The compute runs in hand-written sm_103a CUDA kernels inside ``libaesgb.so``;
``aesgb`` is the thin ctypes binding with the same names as ``include/aesgb.h``.
Importing the package does not load the native library; the first call does,
and fails loudly if it was not built.
"""
__all__ = ["aesgb", "workloads"]
