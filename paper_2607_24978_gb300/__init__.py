"""GB300 (sm_103a) lattice time step of CosmoLattice-style scalar and U(1)-axion
field evolution in an expanding FLRW background.

The compute lives in ``libcl.so`` (CUDA kernels behind the C ABI of
``include/cl.h``); ``cl`` is its Python binding.
"""
from . import build_ext  # noqa: F401
