"""GB300 two-scale finite element hot path (sm_103a CUDA behind a C ABI).

Implements the per-time-step solve of every micro problem of the two-scale
method of Lakkis, Muntean, Richardson and Venkataraman (one micro problem per
macro node on a shared reference cell, coefficients pulled back through the
node's deformation map), the boundary-flux reduction that feeds the macro
source, and the macro solve that closes the coupling iteration.  The C ABI is
declared in ``include/tsfem.h``; :mod:`.binding` mirrors it in Python.
"""
from .binding import *  # noqa: F401,F403
from .binding import TwoScale, ThreeField, TsfError, load_library, LIB_PATH, EXPORTS, EXPORTS3  # noqa: F401
