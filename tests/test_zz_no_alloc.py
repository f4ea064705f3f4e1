"""bmlp_rms_tc_noalloc, the closure entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc: code whose device memory
belongs to a pool allocator or a fixed budget, and latency-critical paths that
cannot take the device synchronisation of an allocation. Its scratch is a
fixed 16 MiB __device__ array shared by every call. This file is collected
last so that a failure here stops a run only after every other test ran.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pkg = pytest.importorskip("paper_2408_10369_gb300")
from paper_2408_10369_gb300 import bmlp  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = ((1000, 1.6, 1, bmlp.BMLP_FMT_U8), (2048, 2.0, 2, bmlp.BMLP_FMT_U8), (777, 1.2, 3, bmlp.BMLP_FMT_PACKED64))


def test_noalloc_matches_oracle_and_bmlp_rms_on_two_calls():
    ctx = pkg.Context(0)
    try:
        for n, d, seed, fmt in CASES:
            ip, ix = wl.er_graph(n, d, seed)
            want = oracle.closure(n, ip, ix)
            want_iters = oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
            dense = wl.dense_u8(n, ip, ix)
            host = dense if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(dense).view(np.int64)
            R = torch.from_numpy(np.ascontiguousarray(host)).cuda()
            ref = torch.zeros_like(R)
            it_ref = ctx.rms(R, n, ref, fmt=fmt, variant="rms_tc")
            for call in range(2):  # two calls in a row share (and reuse) the scratch
                out = torch.full_like(R, 0x55)
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
                it = bmlp.rms_tc_noalloc(R, n, out, fmt=fmt)
                torch.cuda.synchronize()
                free1 = torch.cuda.mem_get_info()[0]
                got = out.cpu().numpy()
                got = got if fmt == bmlp.BMLP_FMT_U8 else wl.unpack_rows(got.view(np.uint64), n)
                assert np.array_equal(got, want), (n, call)
                assert it == want_iters == it_ref, (n, call, it, want_iters, it_ref)
                assert torch.equal(out, ref)
                if call == 1:  # after the first call has set the device up, a call allocates nothing
                    assert free1 == free0, (n, free0, free1)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    n = 2049
    R = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    with pytest.raises(bmlp.BmlpError) as e:
        bmlp.rms_tc_noalloc(R, n, R.clone())
    assert e.value.status == bmlp.BMLP_ERR_UNSUPPORTED


def test_noalloc_rejects_host_memory():
    n = 64
    R = torch.zeros((n, n), dtype=torch.uint8)
    with pytest.raises(bmlp.BmlpError) as e:
        bmlp.rms_tc_noalloc(R, n, R.clone())
    assert e.value.status == bmlp.BMLP_ERR_INVALID_ARG
