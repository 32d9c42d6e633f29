"""GB300-native CheFSI pass of divide-and-conquer Kohn-Sham DFT (arXiv 2609.13115).

The compute path is libxls.so (hand-written sm_103a CUDA behind the C ABI of include/xls.h);
`xls` is its ctypes binding and `build` compiles it in-tree.
"""
from . import xls  # noqa: F401
from .xls import Grid, XlsError, load  # noqa: F401
