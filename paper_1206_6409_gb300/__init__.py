"""GB300 (sm_103a) implementation of the data-parallel hot path of GenCD
(Scherrer, Halappanavar, Tewari, Haglin: "Scaling Up Coordinate Descent
Algorithms for Large l1 Regularization Problems").

The compute path is the CUDA library libgencd.so behind include/gencd.h;
``binding`` is a ctypes marshalling layer over it with the same function
names.  ``build.build()`` compiles the library with nvcc.
"""

from . import binding  # noqa: F401
from .binding import Problem, GencdError, lib  # noqa: F401

__all__ = ["binding", "Problem", "GencdError", "lib"]
