"""GB300-native sparsify-and-sweep preconditioned Lippmann-Schwinger solver.

Liu & Ying, arXiv:1705.09443.  The compute path is the CUDA library liblss.so
(C ABI in include/lss.h); this package only marshals arguments to it.
"""
from ._lib import LSS_FP64, LSS_MIXED, LssError, load  # noqa: F401
from .solver import LSSolver, LSSolverBatch, GmresOptions  # noqa: F401
from .autograd import LSSolve, ls_solve  # noqa: F401
