"""GB300-native patch-based AMR solver for the compressible Euler equations.

The solver is the CUDA library ``_lib/libamr.so`` (sources in ``csrc/``, ABI in
``include/amr.h`` at the repository root); ``amr`` is its Python binding and
``build`` compiles it for sm_103a.
"""
from .amr import AMR, AMRError, load  # noqa: F401
