"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/bmlp.h declares. No compute call is made here."""
import ctypes

import paper_2408_10369_gb300 as pkg


def test_library_exports_every_declared_symbol():
    L = pkg.lib()
    names = pkg.header_functions()
    assert "bmlp_rms" in names and "bmlp_smp" in names and "bmlp_compose" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_options_defaults_and_no_device_error():
    o = pkg.make_options()
    assert o.variant == 0 and o.loop == 0 and o.reflexive == 0
    L = pkg.lib()
    h = ctypes.c_void_p()
    # no CUDA device in this container (or a bad index): a clean error, no crash
    assert L.bmlp_ctx_create(ctypes.byref(h), 1 << 20) == pkg.bmlp.BMLP_ERR_INVALID_ARG
    assert L.bmlp_ctx_destroy(None) == 0
