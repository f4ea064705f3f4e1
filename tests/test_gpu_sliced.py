"""Full frontier closures expanded 64 sources at a time (bit-sliced frontiers).

BMLP_SMP_PACKED closures with n >= 4096 whose first squaring widens the rows
fast (not path-like, no hub columns) run Algorithm 2 for 64 source rows per CTA, with bit j of the
state word of constant w standing for source s0 + j, pulling over the word
index of R^T. Bits against the oracle, the reported level count (deepest BFS
level + 1, as for the one-query-per-warp kernel), ragged batches (n not a
multiple of 64), both formats, the reflexive option, host buffers and the
time budget.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pkg = pytest.importorskip("paper_2408_10369_gb300")
from paper_2408_10369_gb300 import bmlp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graph(kind, n, p, seed):
    if kind == "er":
        return wl.er_graph(n, p, seed)
    if kind == "powerlaw":
        return wl.powerlaw_csr(n, p, 1000, seed)
    return wl.sbm_sparse_csr(n, 8, p / n * 8 * 0.8, p / n * 8 * 0.2 / 7, seed)


# (kind, n, mean degree or exponent, seed, expected path): rows that widen fast (mean degree >= 4) go sliced; sparser
# random graphs and power laws may take either frontier kernel, with the same bits and level count
@pytest.mark.parametrize("kind,n,p,seed,sliced", [("er", 4096, 4.0, 1, True), ("er", 6001, 5.0, 2, True),
                                                  ("er", 5003, 8.0, 3, True), ("sbm", 4161, 6.0, 5, True),
                                                  ("powerlaw", 4500, 2.1, 4, None), ("er", 6001, 1.5, 2, None)])
def test_sliced_closure_matches_oracle(ctx, kind, n, p, seed, sliced):
    ip, ix = graph(kind, n, p, seed)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    lv = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    st = ctx.stats()
    if sliced is not None:
        assert st["sliced_closures"] == int(sliced)
    got = wl.unpack_rows(out.cpu().numpy().view(np.uint64), n)
    want, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32))
    np.testing.assert_array_equal(got, want)
    assert lv == int(depth.max()) + 1


def test_sliced_u8_reflexive_and_host_buffers(ctx):
    n = 4300
    ip, ix = wl.er_graph(n, 5.0, 6)
    want = oracle.closure(n, ip, ix)
    R = dev(wl.dense_u8(n, ip, ix))
    out = torch.zeros_like(R)
    ctx.rms(R, n, out, fmt=bmlp.BMLP_FMT_U8, variant="smp_packed", reflexive=True)
    torch.cuda.synchronize()
    assert ctx.stats()["sliced_closures"] == 1
    np.testing.assert_array_equal(out.cpu().numpy(), want | np.eye(n, dtype=np.uint8))
    Ph = torch.from_numpy(wl.csr_to_packed(n, ip, ix).view(np.int64)).pin_memory()
    oh = torch.zeros_like(Ph).pin_memory()
    ctx.rms(Ph, n, oh, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(oh.numpy().view(np.uint64), n), want)


def test_path_like_relation_keeps_the_query_kernel(ctx):
    """A chain with 1 % shortcuts is squared first and expanded one query per
    warp: no sliced launch, same bits."""
    n = 5000
    src = np.arange(n - 1)
    a, b = wl.random_pairs(n, 50, 7)
    ip, ix = wl.csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([src + 1, b]))
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["sliced_closures"] == 0 and st["frontier_squarings"] >= 1
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), oracle.closure(n, ip, ix))


def test_sliced_budget_is_reported(ctx):
    """A time budget that runs out stops every batch between levels and the
    call reports BMLP_ERR_BUDGET; the context then closes exactly."""
    n = 16384
    ip, ix = wl.er_graph(n, 5.0, 8)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    with pytest.raises(bmlp.BmlpError) as e:
        ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed", budget_ns=1)
    assert e.value.status == bmlp.BMLP_ERR_BUDGET
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    rows = np.arange(0, n, 97, dtype=np.int32)
    want, _, _ = oracle.reach_rows(n, ip, ix, rows)
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64)[rows], n), want)
