"""GB300-native deflated restarted Lanczos solvers (arXiv:0901.3163).

Lan-DR / MinRes-DR for the first right-hand side and D-CG / D-MinRes for the
rest, on the hermitian Wilson-Dirac operators D^dagger D and gamma5 D, as
hand-written sm_103a CUDA kernels behind the C ABI of include/dlz.h.  The
Python layer (`dlz`) only marshals arguments.
"""
from . import dlz  # noqa: F401  (raises ImportError when libdlz.so is missing)
from .dlz import (  # noqa: F401
    D, DDAG, DDAGD, F32, F64, Q, DlzError, Params, Stats, apply, create_operator, dcg,
    defl_count, defl_get, defl_load, defl_save, dminres, landr, minresdr, params_default,
)
