"""GB300 (sm_103a) library for the adaptively compressed polarizability operator (arXiv:1605.08021).

The compute path is ``libacp.so`` (CUDA kernels behind the C ABI of ``include/acp.h``); this
package holds its build script and a ctypes binding that only marshals arguments.
"""
from .binding import (ACP_METHOD_ACP, ACP_METHOD_PLAIN, ACP_PREC_FP64, ACP_PREC_MIXED, AcpError,  # noqa: F401
                      Context, declared_symbols,
                      batch_dynamical_matrix, grid_supported, load, options, phonon_dos)
