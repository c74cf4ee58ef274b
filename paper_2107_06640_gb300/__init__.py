"""GB300-native ADER-DG solver for the coupled elastic-acoustic wave equation
with a gravitational free surface, rate-2 local time stepping and dynamic
rupture (after Krenz et al., SC'21).

The computation lives in the C-ABI library libadg.so (include/adg.h): CUDA
kernels for sm_103a plus C++ host set-up.  `_lib` is the ctypes binding with
the C names; `Solver` is a convenience wrapper holding one context.
"""

from . import _lib  # noqa: F401
from ._lib import AdgError, ADG_FP32, ADG_FP64, ADG_3XTF32, ADG_FRICTION_LSW, ADG_FRICTION_RS  # noqa: F401
from .solver import Solver, plan  # noqa: F401
