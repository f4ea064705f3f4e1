"""Squarings on bit rows before the tensor cores: the engine switch inside one closure.

For n >= 4096 a tensor-core closure first squares R on word-indexed bit rows
for as long as one such step is predicted to cost less than a tensor-core
product, then hands the squared R to the tensor cores (or stops there when a
step changed nothing). Every step is the same R <- R + R R whichever engine
runs it, so the bits equal the oracle's closure and the number of products
equals the oracle's iteration count ceil(log2 L) + 1 (reading c3), with the
work split between `sparse_squarings` and tensor-core `product_launches`.
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


def shortcut_graph(n, shape, seed):
    if shape == "grid":
        side = int(np.sqrt(n))
        idx = np.arange(n)
        right = idx[(idx % side + 1 < side) & (idx + 1 < n)]
        down = idx[idx + side < n]
        src, dst = np.concatenate([right, down]), np.concatenate([right + 1, down + side])
    else:
        src = np.arange(n - 1)
        dst = src + 1
    a, b = wl.random_pairs(n, max(1, round(0.01 * n)), seed)
    return wl.csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([dst, b]))


def graph(kind, n, p, seed):
    if kind == "er":
        return wl.er_graph(n, p, seed)
    if kind == "powerlaw":
        return wl.powerlaw_csr(n, p, 1000, seed)
    return shortcut_graph(n, kind, seed)


def closure_packed(ctx, n, ip, ix, **kw):
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    it = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc", **kw)
    torch.cuda.synchronize()
    return wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), it, ctx.stats()


# ragged sizes (not multiples of 64 / 128 / 256), sparse-to-dense random graphs, skewed degrees and long paths
CASES = [("er", 9001, 1.5, 1), ("er", 8300, 4.0, 2), ("powerlaw", 9000, 2.1, 3), ("chain", 9500, 0, 4),
         ("grid", 10100, 0, 5)]


@pytest.mark.parametrize("kind,n,p,seed", CASES)
def test_switch_matches_oracle_and_iteration_count(ctx, kind, n, p, seed):
    ip, ix = graph(kind, n, p, seed)
    want = oracle.closure(n, ip, ix)
    got, it, st = closure_packed(ctx, n, ip, ix)
    np.testing.assert_array_equal(got, want)
    assert st["sparse_squarings"] >= 1
    assert st["sparse_squarings"] + st["product_launches"] + st["thin_squarings"] == it
    assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    # every squaring on the tensor cores: the same bits and the same count
    got2, it2, st2 = closure_packed(ctx, n, ip, ix, tc_only=True)
    np.testing.assert_array_equal(got2, want)
    assert st2["sparse_squarings"] == st2["thin_squarings"] == 0 and st2["product_launches"] == it2 == it


def test_fixpoint_reached_on_bit_rows(ctx):
    """A sparse relation with short paths: every squaring stays on bit rows,
    the tensor cores never run, and the last step is the no-change check."""
    n = 12000
    ip, ix = wl.er_graph(n, 0.4, 6)
    got, it, st = closure_packed(ctx, n, ip, ix)
    np.testing.assert_array_equal(got, oracle.closure(n, ip, ix))
    assert st["product_launches"] == 0
    assert st["sparse_squarings"] == it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))


@pytest.mark.parametrize("d", [0.4, 2.0])
def test_switch_u8_reflexive(ctx, d):
    """u8 matrices and I + R1+, through both exits (fixpoint on bit rows at
    d = 0.4, hand-over to the tensor cores at d = 2)."""
    n = 8250
    ip, ix = wl.er_graph(n, d, 7)
    R = dev(wl.dense_u8(n, ip, ix))
    out = torch.zeros_like(R)
    ctx.rms(R, n, out, fmt=bmlp.BMLP_FMT_U8, variant="rms_tc", reflexive=True)
    torch.cuda.synchronize()
    want = oracle.closure(n, ip, ix)
    np.fill_diagonal(want, 1)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    st = ctx.stats()
    assert st["sparse_squarings"] >= 1
    assert (st["product_launches"] == 0) == (d < 1)


def test_switch_host_buffers(ctx):
    """Host (pinned) input and output: staged by the library, same bits."""
    n = 8400
    ip, ix = wl.er_graph(n, 1.5, 8)
    P = torch.from_numpy(wl.csr_to_packed(n, ip, ix).view(np.int64)).pin_memory()
    out = torch.zeros_like(P).pin_memory()
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(out.numpy().view(np.uint64), n), oracle.closure(n, ip, ix))
    assert ctx.stats()["sparse_squarings"] >= 1


def test_switch_iteration_cap(ctx):
    """A cap below the needed products gives BMLP_ERR_NOT_CONVERGED with and
    without the switch (the bit-row steps count against the cap)."""
    n = 9000
    ip, ix = shortcut_graph(n, "chain", 9)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    for tc_only in (False, True):
        with pytest.raises(bmlp.BmlpError) as e:
            ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc", max_iters=3, tc_only=tc_only)
        assert e.value.status == bmlp.BMLP_ERR_NOT_CONVERGED
    # the context is usable afterwards
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), oracle.closure(n, ip, ix))


@pytest.mark.parametrize("d2", [0.4, 2.0])
def test_compose_switch(ctx, d2):
    """(I + R2+) R1 with R2+ started on bit rows: every row against the oracle."""
    n = 8320
    csr1 = wl.er_graph(n, 1.0, 10)
    csr2 = wl.er_graph(n, d2, 11)
    A = dev(wl.csr_to_packed(n, *csr1).view(np.int64))
    B = dev(wl.csr_to_packed(n, *csr2).view(np.int64))
    out = torch.zeros_like(A)
    ctx.compose(A, B, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc")
    torch.cuda.synchronize()
    assert ctx.stats()["sparse_squarings"] >= 1
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n),
                                  oracle.compose_rows(n, csr1, csr2))


# ------------------------------------------------ Algorithm 1 as printed --
def offdiag_L0(n, ip, ix):
    """Longest shortest path between two different constants (BFS distances from scipy)."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(len(ix)), ix, ip), shape=(n, n))
    D = csgraph.shortest_path(A, method="D", unweighted=True)
    np.fill_diagonal(D, 0)
    fin = D[np.isfinite(D)]
    return int(fin.max()) if fin.size else 0


@pytest.mark.parametrize("fmt", ["u8", "packed"])
@pytest.mark.parametrize("n,d,seed", [(1, 0.0, 0), (2, 1.0, 1), (65, 1.3, 2), (300, 1.1, 3), (1000, 2.0, 4),
                                      (2500, 1.2, 5)])
def test_alg1_literal_form(ctx, fmt, n, d, seed):
    """(I + R1)^(2^k) R1 through bmlp_rms_alg1: the closure's bits, and
    squarings + 1 products with the squarings fixed by L0."""
    ip, ix = wl.er_graph(n, d, seed)
    want = oracle.closure(n, ip, ix)
    if fmt == "u8":
        R = dev(wl.dense_u8(n, ip, ix))
        out = torch.zeros_like(R)
        it = ctx.rms_alg1(R, n, out, fmt=bmlp.BMLP_FMT_U8)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    else:
        R = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
        out = torch.zeros_like(R)
        it = ctx.rms_alg1(R, n, out, fmt=bmlp.BMLP_FMT_PACKED64)
        torch.cuda.synchronize()
        got = wl.unpack_rows(out.cpu().numpy().view(np.uint64), n)
    np.testing.assert_array_equal(got, want)
    assert it == oracle.alg1_products(offdiag_L0(n, ip, ix))


def test_alg1_self_loop_and_reflexive(ctx):
    for loop in (0, 1):
        R = torch.tensor([[loop]], dtype=torch.uint8, device="cuda")
        out = torch.zeros_like(R)
        assert ctx.rms_alg1(R, 1, out) == 2
        assert int(out.item()) == loop
    n = 700
    ip, ix = wl.er_graph(n, 1.4, 12)
    R = dev(wl.dense_u8(n, ip, ix))
    out = torch.zeros_like(R)
    ctx.rms_alg1(R, n, out, reflexive=True)
    want = oracle.closure(n, ip, ix)
    np.fill_diagonal(want, 1)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    with pytest.raises(bmlp.BmlpError) as e:
        ctx.rms_alg1(R, n, out, variant="smp_packed")
    assert e.value.status == bmlp.BMLP_ERR_INVALID_ARG


def test_alg1_large_dag_with_bit_row_start(ctx):
    """n = 9,000 DAG (forward chain plus forward shortcuts, so L0 = L): the
    squarings start on bit rows; bits and the product count against the oracle."""
    n = 9000
    a, b = wl.random_pairs(n, 90, 13)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    src = np.concatenate([np.arange(n - 1), lo[keep]])
    dst = np.concatenate([np.arange(1, n), hi[keep]])
    ip, ix = wl.csr_from_pairs(n, src, dst)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    it = ctx.rms_alg1(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64)
    torch.cuda.synchronize()
    assert ctx.stats()["sparse_squarings"] >= 1
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), oracle.closure(n, ip, ix))
    assert it == oracle.alg1_products(oracle.longest_shortest_path(n, ip, ix))


# Once a 4-bit squaring has made R nearly its closure, a squaring runs only on the rows and columns that still hold
# zeros (columns with fewer than n / 2 ones, and the rows with a zero elsewhere), on bit rows: same bits, same count.
@pytest.mark.parametrize("n,d,seed", [(12000, 4.0, 31), (20001, 2.5, 32)])
def test_squaring_on_zero_rows_and_columns(ctx, n, d, seed):
    ip, ix = wl.er_graph(n, d, seed)
    want = oracle.closure(n, ip, ix)
    got, it, st = closure_packed(ctx, n, ip, ix)
    np.testing.assert_array_equal(got, want)
    assert st["thin_squarings"] >= 1
    assert st["sparse_squarings"] + st["product_launches"] + st["thin_squarings"] == it
    assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))


def test_zero_rows_and_columns_that_fill_in():
    """A dense random part with a 60-node chain hanging off it: the chain's columns are reached by most rows only
    after several squarings, so squarings restricted to the rows and columns holding zeros find new ones (here in
    u8 and with I + R1+ as well)."""
    c = pkg.Context(0)
    try:
        n0, tail = 9000, 60
        n = n0 + tail
        ip0, ix0 = wl.er_graph(n0, 5.0, 33)
        src = np.concatenate([np.repeat(np.arange(n0), np.diff(ip0)), [0], n0 + np.arange(tail - 1)])
        dst = np.concatenate([ix0, [n0], n0 + 1 + np.arange(tail - 1)])
        ip, ix = wl.csr_from_pairs(n, src, dst)
        want = oracle.closure(n, ip, ix)
        got, it, st = closure_packed(c, n, ip, ix)
        np.testing.assert_array_equal(got, want)
        assert st["thin_squarings"] >= 1
        assert st["sparse_squarings"] + st["product_launches"] + st["thin_squarings"] == it
        assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
        R = dev(wl.dense_u8(n, ip, ix))
        out = torch.zeros_like(R)
        c.rms(R, n, out, fmt=bmlp.BMLP_FMT_U8, variant="rms_tc", reflexive=True)
        torch.cuda.synchronize()
        np.fill_diagonal(want, 1)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
    finally:
        c.close()
