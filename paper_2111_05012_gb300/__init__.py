"""GB300 (sm_103a) adaptive-multigrid solver for the Wilson-clover Dirac
equation (arXiv:2111.05012), behind the C ABI of include/lqcd_amg.h.

``capi`` is the ctypes binding (same names as the C entry points);
``build`` compiles libamg.so in-tree with nvcc.
"""
from . import capi  # noqa: F401
