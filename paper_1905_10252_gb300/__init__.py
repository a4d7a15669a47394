"""GB300-native hot path of the SMC sampler of Varsi et al. (arXiv:1905.10252).

The compute path lives in ``csrc/`` (hand-written sm_103a CUDA behind a C-ABI,
``libsmc.so``); ``native`` is the thin ctypes binding with the same names as the
C entry points.  Importing the package loads nothing: ``native.lib()`` loads the
library on first use and raises if it has not been built.
"""
__all__ = ["native", "inputs"]
