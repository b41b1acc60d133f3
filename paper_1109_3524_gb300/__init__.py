"""GB300 immersed-boundary projection library (Python binding of libibm.so).

The CUDA library does the work; this package only marshals arguments and lets
PyTorch own the device workspace and the stream.  Importing it does not load
the library; constructing a ``Sim`` does, and fails loudly if it is missing.
"""
from ._abi import (IBM_BC_FREESTREAM, IBM_BC_WALLS, IBM_PREC_FP64, IBM_PREC_MIXED,  # noqa: F401
                   IBM_PRECOND_AMG, IBM_PRECOND_JACOBI, IBM_PRECOND_SCHUR, IBM_PRECOND_NONE, IBM_WARM_PREV,
                   IBM_WARM_ZERO, IBM_WARM_EXTRAP, IBM_WARM_CNN, IBM_WARM_PROJ, LIB_PATH, SIGNATURES, load)
from .sim import Config, HostCtx, IbmError, Sim, Unet, create_host_only  # noqa: F401
from . import warmstart  # noqa: F401
