"""Failure detection without a GPU fault: every in-kernel wait is bounded.

A call with a one-nanosecond wait bound cannot finish its pipeline waits, so
the kernel records an error word, drains its own copies and MMAs, frees its
TMEM and returns; the host reports BMLP_ERR_TIMEOUT and the context (and the
GPU) stays usable for the next call. A time budget that runs out is reported
as BMLP_ERR_BUDGET the same way."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pkg = pytest.importorskip("paper_2408_10369_gb300")
from paper_2408_10369_gb300 import bmlp  # noqa: E402

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_context_recovers():
    ctx = pkg.Context(0)
    try:
        n = 1500
        ip, ix = wl.er_graph(n, 2.0, 9)
        R = torch.from_numpy(wl.dense_u8(n, ip, ix)).cuda()
        src = torch.from_numpy(wl.query_rows(n, 300, 1, 8, 9).view(np.int64)).cuda()
        out = torch.zeros_like(src)
        with pytest.raises(bmlp.BmlpError) as e:
            ctx.smp(R, n, src, 300, out, variant="smp_tc", timeout_ns=1)
        assert e.value.status == bmlp.BMLP_ERR_TIMEOUT
        # the same context, normal bounds: exact results again
        ctx.smp(R, n, src, 300, out, variant="smp_tc")
        torch.cuda.synchronize()
        want, _ = oracle.smp(n, ip, ix, src.cpu().numpy().view(np.uint64))
        np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want)
        o2 = torch.zeros_like(R)
        ctx.rms(R, n, o2, variant="rms_tc")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o2.cpu().numpy(), oracle.closure(n, ip, ix))
    finally:
        ctx.close()


def _chain_with_shortcuts(n, seed):
    src = np.arange(n - 1)
    a, b = wl.random_pairs(n, max(1, n // 100), seed)
    return wl.csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([src + 1, b]))


@pytest.mark.parametrize("case", ["dense_e2m1_pairs", "sparse_e4m3_clusters"])
def test_squaring_wait_timeout_recovers(case):
    """The 4-bit 2-SM squaring kernel (dense input) and the E4M3 cluster
    kernel with block skipping (block-sparse input): a one-nanosecond wait
    bound gives BMLP_ERR_TIMEOUT, and the same context then closes exactly."""
    ctx = pkg.Context(0)
    try:
        if case == "dense_e2m1_pairs":
            n = 1500
            ip, ix = wl.er_graph(n, 3.0, 19)
        else:
            n = 3000
            ip, ix = _chain_with_shortcuts(n, 20)
        R = torch.from_numpy(wl.dense_u8(n, ip, ix)).cuda()
        out = torch.zeros_like(R)
        with pytest.raises(bmlp.BmlpError) as e:
            ctx.rms(R, n, out, variant="rms_tc", timeout_ns=1)
        assert e.value.status == bmlp.BMLP_ERR_TIMEOUT
        ctx.rms(R, n, out, variant="rms_tc")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.closure(n, ip, ix))
        st = ctx.stats()
        if case == "dense_e2m1_pairs":
            assert st["e2m1_products"] == st["product_launches"]
        else:
            assert st["e2m1_products"] < st["product_launches"]
    finally:
        ctx.close()
