"""GB300-native (sm_103a) Boolean Matrix Logic Programming.

Bottom-up evaluation of linear dyadic recursive datalog as Boolean matrix
algebra (BMLP-RMS, BMLP-SMP and two-relation composition) in hand-written
CUDA behind the C ABI of ``include/bmlp.h``; ``bmlp`` is its Python binding.
"""
from .bmlp import (BMLP_FMT_PACKED64, BMLP_FMT_U8, BMLP_LOOP_GRAPH, BMLP_LOOP_HOST, BmlpError, Context,  # noqa: F401
                   header_functions, lib, library_path, make_options)
