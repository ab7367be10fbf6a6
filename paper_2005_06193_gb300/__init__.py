"""GB300-native (sm_103a) EGFEM Newton hot path.

The compute path is the CUDA library built from ``csrc/`` (C ABI in include/egfem.h);
``egfem`` is its thin ctypes binding and ``autograd`` wraps the adjoint in a
``torch.autograd.Function``.
"""
from .egfem import (G_EXP, G_GRADPOW, G_NONE, G_POW, ITER_NEWTON, ITER_PICARD, OP_CSF, OP_MATRIX_FREE, PREC_FP64,  # noqa: F401
                    PREC_MIXED, BatchHandle,
                    EgfemError, Handle, default_options, inspect_tensor, lib, make_problem,
                    selftest_grid_barrier, W_LAGRANGE, W_QUADRATURE)
