"""GB300-native density-fitted self-consistent GW (single GPU, sm_103a).

The method runs in the CUDA kernels of libgwgb.so (C ABI in include/gwgb.h);
`GW` is the Python binding.  Importing this package does not load the
library; constructing a `GW` does, and fails loudly when it is missing.
"""
from .gw import GW, GWError, load, LIB_PATH, QUANTITIES

__all__ = ["GW", "GWError", "load", "LIB_PATH", "QUANTITIES"]
