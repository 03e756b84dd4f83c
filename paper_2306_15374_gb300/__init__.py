"""GB300-native LeCo: learned serial-correlation compression of integer columns (arXiv 2306.15374).

The compute path is the CUDA library libleco.so (kernels for sm_103a behind the C ABI declared in
include/leco.h); this package holds its sources (csrc/), the in-tree build (builder.py) and the
ctypes binding (leco.py).
"""
from .builder import build  # noqa: F401
from .leco import *  # noqa: F401,F403
from .leco import Column, LecoError, PartitionPolicy, fixed, variable  # noqa: F401
