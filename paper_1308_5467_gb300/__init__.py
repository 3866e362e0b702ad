"""GB300-native Kernel Polynomial Method for the density of states.

The compute path lives in libdos.so (hand-written sm_103a CUDA kernels behind
the C ABI of include/dos.h); ``paper_1308_5467_gb300.dos`` is its ctypes
binding.  Build with ``python -m paper_1308_5467_gb300.build``.
"""
__all__ = ["dos", "build"]
