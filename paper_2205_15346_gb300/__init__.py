"""GB300-native restarted Krylov time evolution exp(-iHt)v (arXiv 2205.15346).

The compute path is libte (CUDA for sm_103a, C ABI in include/te.h); ``te`` is
its ctypes binding.  Importing this package does not load the library; the first
call into ``te`` does, and fails loudly if libte.so has not been built.
"""
from . import te  # noqa: F401

__all__ = ["te"]
