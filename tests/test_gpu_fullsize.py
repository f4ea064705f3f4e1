"""The five workload configurations at full size, through the C ABI, in the
launch configurations bench.py uses, every output bit against the oracle
(large closures as LSB-first 64-bit words, 4,096 oracle rows at a time)."""
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


def popcount_rows(packed):
    return np.unpackbits(packed.view(np.uint8), axis=1).sum(1)


def assert_closure_words(n, ip, ix, got):
    """Every bit of the n x n closure `got` (packed rows, uint64) against the
    oracle's bit rows, block by block."""
    for r0, blk in oracle.closure_bits_chunks(n, ip, ix, 4096):
        part = got[r0:r0 + blk.shape[0], :blk.shape[1]]
        if not np.array_equal(part, blk):
            bad = r0 + np.nonzero((part != blk).any(axis=1))[0]
            raise AssertionError("n = %d: %d rows differ, first %s" % (n, len(bad), bad[:5].tolist()))


def u8_to_words(m):
    pk = np.packbits(m != 0, axis=1, bitorder="little")
    w = wl.words(m.shape[1])
    pk = np.pad(pk, ((0, 0), (0, 8 * w - pk.shape[1])))
    return np.ascontiguousarray(pk).view(np.uint64)


def test_config1_er2000(ctx):
    """n = 2,000, p = 2/n: RMS on every variant and SMP from 16 random sources."""
    n = 2000
    ip, ix = wl.er_csr(n, 2.0 / n, 0)
    R = dev(wl.dense_u8(n, ip, ix))
    want = oracle.closure(n, ip, ix)
    L = oracle.longest_shortest_path(n, ip, ix)
    for v in ("rms_tc", "rms_packed", "smp_packed", "smp_tc"):
        out = torch.zeros_like(R)
        it = ctx.rms(R, n, out, variant=v)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        if v.startswith("rms"):
            assert it == oracle.rms_iterations(L)
    src = wl.query_rows(n, 1, 16, 16, 0)
    want_q, _ = oracle.smp(n, ip, ix, src)
    for v in ("smp_packed", "smp_tc"):
        out = torch.zeros((1, src.shape[1]), dtype=torch.int64, device="cuda")
        ctx.smp(R, n, dev(src.view(np.int64)), 1, out, variant=v)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want_q)


@pytest.mark.parametrize("n", [8192, 16384, 32768])
@pytest.mark.parametrize("d", [1.5, 4.0])
def test_config2_er_tensor_cores(ctx, n, d):
    """Packed rows in and out (the bench.py default) and u8 in and out: every
    bit of both closures, and the product count."""
    ip, ix = wl.er_graph(n, d, 0)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    it = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc")
    torch.cuda.synchronize()
    assert_closure_words(n, ip, ix, out.cpu().numpy().view(np.uint64))
    _, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32), want_rows=False)
    assert it == oracle.rms_iterations(int(depth.max()))
    del P, out
    R = dev(wl.dense_u8(n, ip, ix))
    out8 = torch.zeros_like(R)
    it8 = ctx.rms(R, n, out8, variant="rms_tc")
    torch.cuda.synchronize()
    assert it8 == it
    assert_closure_words(n, ip, ix, u8_to_words(out8.cpu().numpy()))


def test_largest_tensor_core_closure(ctx):
    """n = 65,536 (beyond the block-map limit of 256 x 256 blocks, so every
    tensor-core squaring runs on 4-bit operands; the first ones run on bit
    rows while R is sparse): every bit against the oracle."""
    n = 65536
    ip, ix = wl.er_graph(n, 1.5, 3)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    it = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc")
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["e2m1_products"] == st["product_launches"] >= 1
    assert st["sparse_squarings"] + st["product_launches"] + st["thin_squarings"] == it
    got = out.cpu().numpy().view(np.uint64)
    del P, out
    _, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32), want_rows=False)
    assert it == oracle.rms_iterations(int(depth.max()))
    assert_closure_words(n, ip, ix, got)


@pytest.mark.parametrize("d", [1.5, 4.0])
def test_config2_er8192_packed_and_frontier(ctx, d):
    """The bit-row squaring and frontier variants at n = 8,192: every bit."""
    n = 8192
    ip, ix = wl.er_graph(n, d, 0)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    for v in ("rms_packed", "smp_packed", "smp_tc"):
        out = torch.zeros_like(P)
        ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant=v)
        torch.cuda.synchronize()
        assert_closure_words(n, ip, ix, out.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("variant", ["smp_packed", "smp_tc"])
def test_config3_powerlaw_queries(ctx, variant):
    """n = 65,536 power law, 4,096 query rows of 1-64 sources: every bit."""
    n, q = 65536, 4096
    ip, ix = wl.powerlaw_csr(n, 2.1, 1000, 0)
    P = dev(wl.pack_rows(wl.dense_u8(n, ip, ix)).view(np.int64))
    src = wl.query_rows(n, q, 1, 64, 0)
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    lv = ctx.smp(P, n, dev(src.view(np.int64)), q, out, fmt=bmlp.BMLP_FMT_PACKED64, variant=variant)
    torch.cuda.synchronize()
    want, levels = oracle.smp(n, ip, ix, src)
    got = out.cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(got, wl.pack_rows(want))
    assert lv == int(levels.max()) + 1


def test_config4_kg_batch(ctx):
    """15,000 entities, 1,345 relations, 483,000 triples; every relation's
    closure and 200 two-relation programs in one grouped batch: every bit."""
    rels = wl.kg_relations()
    items, keep, expect = [], [], []
    for r in rels:
        n = r["n"]
        R = dev(wl.pack_rows(wl.dense_u8(n, r["indptr"], r["indices"])).view(np.int64))
        out = torch.zeros_like(R)
        keep += [R, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=bmlp.BMLP_FMT_PACKED64))
        expect.append(("closure", n, r["indptr"], r["indices"]))
    for a, b in wl.kg_compose_pairs(rels, 200, 0):
        n, ents, c1, c2 = wl.union_space(rels[a], rels[b])
        R1 = dev(wl.pack_rows(wl.dense_u8(n, *c1)).view(np.int64))
        R2 = dev(wl.pack_rows(wl.dense_u8(n, *c2)).view(np.int64))
        out = torch.zeros_like(R1)
        keep += [R1, R2, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=n, R1=R1, R2=R2, out=out, fmt=bmlp.BMLP_FMT_PACKED64))
        expect.append(("compose", n, c1, c2))
    iters = ctx.batch_run(items)
    torch.cuda.synchronize()
    # one graph launch for all 1,545 programs (the large ones as device-driven pipelines): one host wait
    assert ctx.stats()["host_syncs"] == 1
    for it, ex, k in zip(items, expect, iters):
        n = ex[1]
        got = it["out"].cpu().numpy().view(np.uint64)
        if ex[0] == "closure":
            want = oracle.closure(n, ex[2], ex[3])
        else:
            want = oracle.compose_rows(n, ex[2], ex[3])
        np.testing.assert_array_equal(got, wl.pack_rows(want))
