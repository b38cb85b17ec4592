"""GB300-native COLA particle-mesh library (ICE-COLA, arXiv:1509.04685).

The compute path is the CUDA library ``_build/libcola_gb300.so`` (C ABI in
``include/cola.h``); this package is its ctypes binding plus small helpers
that allocate torch tensors for the state and the workspace.  Importing it
fails loudly if the library has not been built.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import LIB, LIB_PATH  # noqa: F401
from .sim import Simulation  # noqa: F401
