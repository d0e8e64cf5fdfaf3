"""GB300 (sm_103a) symmetric fast multipole gravity with adaptive kernel
softening: a C-ABI CUDA library (``csrc/``, ``include/sfmm.h``) and its thin
ctypes binding (``sfmm``)."""
from . import sfmm  # noqa: F401
from .sfmm import Solver  # noqa: F401

__all__ = ["sfmm", "Solver"]
