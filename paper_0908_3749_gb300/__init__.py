"""GB300 (sm_103a) implementation of the hot path of the energy-conserving
MRT finite-difference lattice Boltzmann model for compressible flow
(Chen, Xu, Zhang, Li; D2V16).

The compute runs in hand-written CUDA kernels behind the C ABI of
``include/lbm.h`` (library ``_build/liblbm.so``); ``lbm`` is its ctypes
binding.
"""
from . import lbm  # noqa: F401
