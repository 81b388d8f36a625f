"""GB300 (sm_103a) D2Q9 multi-relaxation-time lattice Boltzmann library.

The compute path is liblbm.so (CUDA, include/lbm.h); ``lbm`` is its thin
ctypes binding and ``build`` compiles it in-tree.
"""
from . import lbm  # noqa: F401
