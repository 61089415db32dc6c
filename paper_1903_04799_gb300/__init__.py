"""GB300-native lattice Boltzmann squirmers (Kuron et al., arXiv:1903.04799).

The compute path is the CUDA library ``liblbsq.so`` (C ABI in
``include/lbsq.h``); ``lbsq`` is its thin Python binding.
"""
from . import lbsq  # noqa: F401
from .lbsq import Lattice  # noqa: F401

__all__ = ["lbsq", "Lattice"]
