"""GB300-native augmented-Lagrangian multigrid for variable-viscosity Stokes flow.

The solver lives in the CUDA library libalstokes.so (C ABI in include/alstokes.h);
this package holds its sources (csrc/), its in-tree build (build.py) and a thin
ctypes binding (alstokes.py).
"""
from . import alstokes  # noqa: F401
from .alstokes import ALSError, Batch, Context, load  # noqa: F401
