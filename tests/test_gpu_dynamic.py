"""Incremental closure (bmlp_insert) for a growing database, and the facts
front-end driving the library end to end; bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from golden_io import matrix, read_facts
from paper_2408_10369_gb300 import facts as F

pkg = pytest.importorskip("paper_2408_10369_gb300")

pytestmark = pytest.mark.gpu

PACKED = pkg.BMLP_FMT_PACKED64


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def new_facts(n, m, seed, ip, ix):
    """m new pairs: random ones, a self-loop, a duplicate, and a fact already in R."""
    a, b = wl.random_pairs(n, m, seed)
    e = np.stack([a, b], 1).astype(np.int32)
    extra = [[3 % n, 3 % n], [int(e[0, 0]), int(e[0, 1])]]
    if len(ix):
        extra.append([0 if ip[1] > 0 else int(np.argmax(np.diff(ip) > 0)), int(ix[0])])
    return np.concatenate([e, np.array(extra, np.int32)])


def union_csr(n, ip, ix, e):
    src = np.repeat(np.arange(n), np.diff(ip))
    return wl.csr_from_pairs(n, np.concatenate([src, e[:, 0]]), np.concatenate([ix, e[:, 1]]))


@pytest.mark.parametrize("n,d,m,seed", [(1, 0.0, 1, 0), (130, 0.6, 20, 1), (700, 0.9, 60, 2), (1500, 0.5, 200, 3)])
@pytest.mark.parametrize("fmt", ["u8", "packed"])
def test_insert_matches_recompute(ctx, n, d, m, seed, fmt):
    ip, ix = wl.er_graph(n, d, seed)
    e = new_facts(n, m, seed + 100, ip, ix)
    want = oracle.closure(n, *union_csr(n, ip, ix, e))
    R = wl.dense_u8(n, ip, ix)
    if fmt == "u8":
        C = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
        ctx.rms(dev(R), n, C, variant="rms_tc")
        ctx.insert(C, n, dev(e))
        got = C.cpu().numpy()
    else:
        C = torch.zeros((n, wl.words(n)), dtype=torch.int64, device="cuda")
        ctx.rms(dev(wl.pack_rows(R).view(np.int64)), n, C, fmt=PACKED, variant="smp_packed")
        ctx.insert(C, n, e, fmt=PACKED)                     # facts in host memory
        got = wl.unpack_rows(C.cpu().numpy().view(np.uint64), n)
    np.testing.assert_array_equal(got, want)


def test_insert_host_closure_and_one_by_one(ctx):
    n = 400
    ip, ix = wl.er_graph(n, 0.8, 7)
    e = new_facts(n, 30, 8, ip, ix)
    C = np.zeros((n, n), np.uint8)
    ctx.rms(wl.dense_u8(n, ip, ix), n, C)
    D = C.copy()
    ctx.insert(C, n, e)                                        # host closure buffer
    for k in range(len(e)):
        ctx.insert(D, n, e[k:k + 1])
    want = oracle.closure(n, *union_csr(n, ip, ix, e))
    np.testing.assert_array_equal(C, want)
    np.testing.assert_array_equal(D, want)


def test_insert_rejects_unknown_constants(ctx):
    n = 50
    C = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    before = C.clone()
    with pytest.raises(pkg.BmlpError) as ex:
        ctx.insert(C, n, np.array([[1, 2], [3, 50]], np.int32))
    assert ex.value.status == pkg.BMLP_ERR_INVALID_ARG
    assert torch.equal(C, before)
    ctx.insert(C, n, np.zeros((0, 2), np.int32))           # no facts: no-op


def test_insert_full_size_place_hierarchy(ctx):
    """hasPlace over the 14,541-entity hierarchy, then 300 new contains facts;
    300 sampled rows against the oracle's closure of the grown relation."""
    n = 14541
    (ci, cx), _ = wl.geo_kg(n=n)
    C = dev(wl.csr_to_packed(n, ci, cx).view(np.int64))
    H = torch.zeros_like(C)
    ctx.rms(C, n, H, fmt=PACKED)
    e = new_facts(n, 300, 77, ci, cx)
    ctx.insert(H, n, dev(e), fmt=PACKED)
    got = wl.unpack_rows(H.cpu().numpy().view(np.uint64), n)
    uip, uix = union_csr(n, ci, cx, e)
    rows = np.random.default_rng(5).choice(n, 300, replace=False).astype(np.int32)
    want, _, _ = oracle.reach_rows(n, uip, uix, rows)
    np.testing.assert_array_equal(got[rows], want)


def test_front_end_is_foreign(ctx):
    """Prolog facts in, isForeign facts out, through the library."""
    text = """contains(t1, g2). contains(g3, t1). adjoins(g3, g4).
              location(g1). location(g2). location(g3). location(g4). location(t1). location(t2). location(t3)."""
    f = F.parse_facts(text)
    dom = F.Domain.of(f)
    n = len(dom)
    out = np.zeros((n, n), np.uint8)
    ctx.is_foreign(F.relation_matrix(f["contains"], dom), F.relation_matrix(f["adjoins"], dom), n, out,
                   location=F.type_vector(f["location"], dom))
    got = set(F.matrix_facts("isForeign", out, dom))
    consts, golden = read_facts("p3p5_isforeign.txt")
    assert dom.names == consts
    want = {"isForeign(%s, %s)." % (a, b) for a in consts for b in consts} - \
           {"isForeign(%s, %s)." % p for p in golden["not_isForeign"]}
    assert got == want and len(got) == 45
