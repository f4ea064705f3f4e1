"""GB300-native (sm_103a) Boolean Matrix Logic Programming.

Bottom-up evaluation of linear dyadic recursive datalog as Boolean matrix
algebra (BMLP-RMS, BMLP-SMP and two-relation composition) in hand-written
CUDA behind the C ABI of ``include/bmlp.h``; ``bmlp`` is its Python binding.
"""
from .bmlp import (BMLP_ERR_BUDGET, BMLP_ERR_INVALID_ARG, BMLP_ERR_NOT_CONVERGED, BMLP_ERR_TIMEOUT,  # noqa: F401
                   BMLP_ERR_UNSUPPORTED, BMLP_FMT_PACKED64, BMLP_FMT_U8, BMLP_LOOP_GRAPH, BMLP_LOOP_HOST, BMLP_OK,
                   BmlpError, Context, header_functions, lib, library_path, make_options)
