"""GB300-native windowed median/MAD broadband RFI excision (Buch et al., Section II-D).

The computation lives in librfi.so (hand-written sm_103a CUDA behind the C ABI of
include/rfi.h); this package is its ctypes binding.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import LIB, LIB_PATH, CopiesPlan, Plan, RfiError, Server, check, make_desc  # noqa: F401
