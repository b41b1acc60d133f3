"""CPU oracle (test infrastructure).

Plain FP64 NumPy/SciPy implementation of the immersed-boundary projection
method with direct sparse solves.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library.
"""
from .ibpm import (Grid, Boundary, Oracle, StepStats, roma_delta, mass_diag,  # noqa: F401
                   laplacian, laplacian_bc, gradient, divergence_full,
                   interpolation_E, convection, freestream_boundary,
                   wall_boundary, convective_outflow, pin_matrix)
