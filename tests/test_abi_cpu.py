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


def test_struct_layouts_match_the_header(tmp_path):
    """bmlp_options, bmlp_stats and bmlp_problem as the C compiler lays them
    out from include/bmlp.h (gcc on the host) against the ctypes mirrors."""
    import os
    import subprocess

    import pytest

    from paper_2408_10369_gb300 import bmlp

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"bmlp_options": bmlp.bmlp_options, "bmlp_stats": bmlp.bmlp_stats, "bmlp_problem": bmlp.bmlp_problem}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bmlp.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    try:
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("no host C compiler")
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)
