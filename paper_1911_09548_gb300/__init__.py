"""GB300 space-time multigrid for the transient eddy-current equation (arXiv 1911.09548).

The compute path is the C-ABI library libstmg.so (include/st_mg.h: CUDA kernels
for sm_103a plus a C++ host runtime).  This package holds its sources (csrc/), the
build step (_build.py), the ctypes binding (binding.py) and a small convenience
wrapper (solver.py) that keeps buffers in torch CUDA tensors, and the request-loop
wrapper (serving.py, include/st_mg_serve.h).
"""
from .binding import *  # noqa: F401,F403
from .binding import StMgError, lib, exported_symbols  # noqa: F401
from .solver import SpaceTimeSolver  # noqa: F401
from .serving import SpaceTimeServer  # noqa: F401
