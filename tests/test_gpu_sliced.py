"""Frontier expansion 64 rows at a time (bit-sliced frontiers).

BMLP_SMP_PACKED closures with n >= 4096 whose first squaring widens the rows
fast (not path-like, no hub columns), and query batches of >= 64 rows over
such relations, run Algorithm 2 for 64 rows at once, with bit j of the state
word of constant w standing for row s0 + j, pulling over the word index of
R^T: closures one CTA per 64 sources with the state in global memory, query
batches (n <= 65,536) one thread-block cluster per 64 rows with the frontier
in the cluster's shared memory. Bits against the oracle, the reported level
count (deepest BFS level + 1, as for the one-query-per-warp kernel), the
cluster shapes, ragged batches (n or q not a multiple of 64), empty query
rows, both formats, the reflexive option, host buffers and the time budget.
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
    if kind != "powerlaw":
        assert st["cluster_frontiers"] == 0  # columns without hubs: the global-memory kernel
    got = wl.unpack_rows(out.cpu().numpy().view(np.uint64), n)
    want, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32))
    np.testing.assert_array_equal(got, want)
    assert lv == int(depth.max()) + 1


@pytest.mark.parametrize("n,alpha,seed", [(8192, 2.0, 1), (6000, 2.0, 6), (9000, 2.2, 5)])
def test_sliced_closure_skewed_columns(ctx, n, alpha, seed):
    """Power-law closures (preferential-attachment targets: largest column 7-12 times the mean) whose rows widen
    fast run on the cluster kernel with the identity rows as queries: every bit and the level count."""
    ip, ix = wl.powerlaw_csr(n, alpha, 1000, seed)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    lv = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["sliced_closures"] == 1 and st["cluster_frontiers"] == 1
    want, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32))
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want)
    assert lv == int(depth.max()) + 1
    R = dev(wl.dense_u8(n, ip, ix))
    o8 = torch.zeros_like(R)
    ctx.rms(R, n, o8, fmt=bmlp.BMLP_FMT_U8, variant="smp_packed", reflexive=True)
    torch.cuda.synchronize()
    assert ctx.stats()["cluster_frontiers"] == 1
    np.testing.assert_array_equal(o8.cpu().numpy(), want | np.eye(n, dtype=np.uint8))


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


# ------------------------------------------------------------------ larger closures, query batches --
def sample_rows(n, k=257):
    return np.unique(np.linspace(0, n - 1, k).astype(np.int32))


@pytest.mark.parametrize("n,seed", [(16384, 11), (40000, 12), (65536, 13), (66000, 14)])
def test_sliced_closure_large(ctx, n, seed):
    """Closures of 256 to 1,032 batches of 64 sources (several rounds over the CTAs), sampled rows against the
    oracle."""
    ip, ix = wl.er_graph(n, 5.0, seed)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    assert ctx.stats()["sliced_closures"] == 1
    rows = sample_rows(n)
    want, _, _ = oracle.reach_rows(n, ip, ix, rows)
    got = wl.unpack_rows(out.cpu().numpy().view(np.uint64)[rows], n)
    np.testing.assert_array_equal(got, want)
    del P, out


def query_case(n, q, seed, empty=()):
    src = wl.query_rows(n, q, 1, 64, seed)
    src[list(empty)] = 0
    return src


# Cluster shapes (CTA r of a cluster owns a power-of-two chunk of constants; a cluster is widened while the batches
# leave SMs idle): 4 CTAs of 1,024 constants (n = 4,096, one batch), 5 of 1,024 with a ragged last chunk (n = 5,000),
# 5 of 2,048 (n = 9,001), 8 of 1,024 (n = 8,000, 10 batches), 1 CTA of 4,096 (n = 4,096, 154 batches), 2 of 8,192
# (n = 16,384, 80 batches) and 8 of 8,192 (n = 65,536, below).
@pytest.mark.parametrize("kind,n,p,q,seed,reflexive", [("er", 4096, 6.0, 64, 1, False), ("er", 5000, 5.0, 130, 2, True),
                                                       ("er", 9001, 4.0, 200, 3, False),
                                                       ("powerlaw", 5000, 2.1, 100, 4, False),
                                                       ("powerlaw", 8000, 2.1, 640, 5, True),
                                                       ("er", 4096, 6.0, 9800, 6, False),
                                                       ("er", 16384, 4.0, 5120, 7, True)])
def test_sliced_query_batches(ctx, kind, n, p, q, seed, reflexive):
    """Query rows of 1-64 sources (some rows empty), 64 rows per cluster: bits, level count and reflexive rows
    against the oracle; batches of >= 64 rows over a relation that widens its rows fast take the sliced kernel."""
    ip, ix = graph(kind, n, p, seed)
    src = query_case(n, q, seed, empty=(0, q // 2, q - 1))
    want, levels = oracle.smp(n, ip, ix, src)
    if reflexive:
        want = want | wl.unpack_rows(src, n)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.full((q, src.shape[1]), -1, dtype=torch.int64, device="cuda")
    it = ctx.smp(P, n, dev(src.view(np.int64)), q, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed",
                 reflexive=reflexive)
    torch.cuda.synchronize()
    if kind == "er":
        assert ctx.stats()["sliced_closures"] == ctx.stats()["cluster_frontiers"] == 1
    got = out.cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(wl.unpack_rows(got, n), want)
    # the padding bits of every row's last word stay zero
    np.testing.assert_array_equal(got, wl.pack_rows(want))
    assert it == int(levels.max()) + 1


def test_query_batch_powerlaw_full_size(ctx):
    """The selective-query workload: 4,096 rows of 1-64 sources on the n = 65,536 power-law graph (Zipf 2.1
    out-degrees capped at 1,000), every bit and the level count against the oracle, 64 rows per 8-CTA cluster."""
    n, q = 65536, 4096
    ip, ix = wl.powerlaw_csr(n, 2.1, 1000, 0)
    src = wl.query_rows(n, q, 1, 64, 0)
    want, levels = oracle.smp(n, ip, ix, src)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    it = ctx.smp(P, n, dev(src.view(np.int64)), q, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    assert ctx.stats()["cluster_frontiers"] == 1
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), wl.pack_rows(want))
    assert it == int(levels.max()) + 1
    del P, out


def test_query_batch_path_like_keeps_the_query_kernel(ctx):
    """Query rows over a chain with 1 % shortcuts (rows that do not widen): one query per warp, same bits."""
    n, q = 6000, 96
    src0 = np.arange(n - 1)
    a, b = wl.random_pairs(n, 60, 9)
    ip, ix = wl.csr_from_pairs(n, np.concatenate([src0, a]), np.concatenate([src0 + 1, b]))
    src = query_case(n, q, 10)
    want, levels = oracle.smp(n, ip, ix, src)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    it = ctx.smp(P, n, dev(src.view(np.int64)), q, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    assert ctx.stats()["sliced_closures"] == ctx.stats()["cluster_frontiers"] == 0
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want)
    assert it == int(levels.max()) + 1
