"""GB300-native (sm_103a) Interacting Conditional Wavefunction time stepping, arXiv 1805.11169.

The compute path is the CUDA library ``libicwf.so`` (C ABI in include/icwf.h); this package only
marshals arguments to it through ctypes.  Importing fails loudly when the library is missing.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import Icwf, IcwfError, params_from  # noqa: F401
