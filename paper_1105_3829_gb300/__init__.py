"""GB300-native exact running median (hierarchical recursive running median).

The compute path lives in the C-ABI shared library ``libhrm.so`` (CUDA
kernels for sm_103a, see ``csrc/``); ``hrm`` is its thin ctypes binding.
Importing the package does not load the library; ``hrm.lib()`` does, and
fails loudly when it is missing.
"""
__all__ = ["hrm", "inputs"]
