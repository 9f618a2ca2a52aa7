"""FP64 CPU ORACLE -- test infrastructure only.

A plain, slow restatement of the data-space Hessian method (time stepping in
plain C, everything else in numpy, all in float64).  Only tests/, the package
smoke check and the benchmark's CPU-baseline leg may import it.  It shares no
code with the CUDA path and imports nothing from the product package.
"""
from .core import *  # noqa: F401,F403
from .core import Grid, fd_run  # noqa: F401
