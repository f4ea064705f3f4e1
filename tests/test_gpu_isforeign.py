"""The relation operators of Sec. 3.4 (TRANSP, NEG with type literals, union)
and the composed program P3 u P4 u P5 (isForeign) through the C ABI, bit for
bit against the oracle: the paper's 7-constant example, random small
programs in both formats with location subsets, host buffers, and the
14,541-entity place hierarchy at full size on sampled rows.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from golden_io import matrix, read_facts

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


def csr(m):
    r, c = np.nonzero(m)
    ip = np.zeros(m.shape[0] + 1, np.int64)
    np.add.at(ip, r + 1, 1)
    return np.cumsum(ip), c.astype(np.int32)


def packed_dev(m):
    return dev(wl.pack_rows(m).view(np.int64))


def unpacked(t, n):
    return wl.unpack_rows(t.cpu().numpy().view(np.uint64), n)


def loc_vector(loc):
    return wl.pack_rows(loc.reshape(1, -1).astype(np.uint8))[0]


@pytest.mark.parametrize("n", [1, 63, 64, 65, 200, 1000])
def test_operators(ctx, n):
    rng = np.random.default_rng(n)
    a = (rng.random((n, n)) < 0.05).astype(np.uint8)
    b = (rng.random((n, n)) < 0.05).astype(np.uint8)
    rows = (rng.random(n) < 0.6).astype(np.uint8)
    cols = (rng.random(n) < 0.6).astype(np.uint8)
    out = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    ctx.transpose(dev(a), n, out)
    np.testing.assert_array_equal(out.cpu().numpy(), a.T)
    ctx.union(dev(a), dev(b), n, out)
    np.testing.assert_array_equal(out.cpu().numpy(), a | b)
    ctx.negate(dev(a), n, out)
    np.testing.assert_array_equal(out.cpu().numpy(), 1 - a)
    ctx.negate(dev(a), n, out, rows=dev(loc_vector(rows).view(np.int64)), cols=loc_vector(cols))
    np.testing.assert_array_equal(out.cpu().numpy(), rows[:, None] & cols[None, :] & (1 - a))
    # packed rows, output aliasing the input, host buffers
    P = packed_dev(a)
    ctx.negate(P, n, P, fmt=PACKED)
    np.testing.assert_array_equal(unpacked(P, n), 1 - a)
    host_out = np.zeros((n, n), np.uint8)
    ctx.transpose(a, n, host_out)
    np.testing.assert_array_equal(host_out, a.T)


@pytest.mark.parametrize("n,dens", [(257, 0.05), (5000, 0.002), (12001, 0.0002), (3000, 0.6)])
def test_transpose_packed_tiles(ctx, n, dens):
    """TRANSP on packed rows across many transpose tiles (256 rows x 512 columns each; ragged n, sparse and dense):
    every word of the output, padding bits of the last word included, against numpy."""
    rng = np.random.default_rng(n)
    m = int(dens * n * n)
    a = np.zeros((n, n), np.uint8)
    a[rng.integers(0, n, m), rng.integers(0, n, m)] = 1
    P = packed_dev(a)
    out = torch.full_like(P, -1)
    ctx.transpose(P, n, out, fmt=PACKED)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), wl.pack_rows(np.ascontiguousarray(a.T)))


@pytest.mark.parametrize("variant", ["auto", "rms_tc", "rms_packed", "smp_packed", "smp_tc"])
def test_is_foreign_example(ctx, variant):
    consts, facts = read_facts("p3p5_isforeign.txt")
    n = len(consts)
    contains = matrix(consts, facts["contains"])
    adjoins = matrix(consts, facts["adjoins"])
    out = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    ctx.is_foreign(dev(contains), dev(adjoins), n, out, variant=variant)
    got = out.cpu().numpy()
    np.testing.assert_array_equal(1 - got, matrix(consts, facts["not_isForeign"]))
    assert int(got.sum()) == 45


@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed", "smp_packed"])
@pytest.mark.parametrize("n,seed", [(7, 0), (130, 1), (700, 2), (1500, 3)])
def test_is_foreign_random(ctx, variant, n, seed):
    (ci, cx), (ai, ax) = wl.geo_kg(n=n, n_contains=n // 2, n_adjoins=max(1, n // 6), n_roots=max(1, n // 50),
                                   seed=seed)
    rng = np.random.default_rng(seed)
    loc = (rng.random(n) < 0.8).astype(np.uint8)
    want = oracle.is_foreign(n, (ci, cx), (ai, ax), loc)
    cm, am = wl.dense_u8(n, ci, cx), wl.dense_u8(n, ai, ax)
    out = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    it = ctx.is_foreign(dev(cm), dev(am), n, out, location=loc_vector(loc), variant=variant)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    if variant.startswith("rms"):
        assert it[0] == oracle.rms_iterations(oracle.longest_shortest_path(n, ci, cx))
    P = torch.zeros((n, wl.words(n)), dtype=torch.int64, device="cuda")
    ctx.is_foreign(packed_dev(cm), packed_dev(am), n, P, location=dev(loc_vector(loc).view(np.int64)),
                   fmt=PACKED, variant=variant)
    np.testing.assert_array_equal(unpacked(P, n), want)


def test_is_foreign_host_buffers(ctx):
    n = 300
    (ci, cx), (ai, ax) = wl.geo_kg(n=n, n_contains=150, n_adjoins=40, n_roots=6, seed=9)
    want = oracle.is_foreign(n, (ci, cx), (ai, ax))
    out = np.zeros((n, n), np.uint8)
    ctx.is_foreign(wl.dense_u8(n, ci, cx), wl.dense_u8(n, ai, ax), n, out)
    np.testing.assert_array_equal(out, want)


def forest_ipo(n, contains, adjoins):
    """indirectlyPartOf on a forest of places without the closure machinery:
    X is indirectly part of Y iff X or one of its ancestors adjoins Y (either
    direction); ancestors by walking up the unique parent links."""
    ci, cx = contains
    parent = np.full(n, -1, np.int64)
    for p in range(n):
        parent[cx[ci[p]:ci[p + 1]]] = p
    ai, ax = adjoins
    nb = [set() for _ in range(n)]
    for a in range(n):
        for b in ax[ai[a]:ai[a + 1]]:
            nb[a].add(int(b))
            nb[int(b)].add(a)
    rows, cols = [], []
    for x in range(n):
        ys, z = set(), x
        while z >= 0:
            ys |= nb[z]
            z = parent[z]
        rows += [x] * len(ys)
        cols += sorted(ys)
    return np.array(rows, np.int64), np.array(cols, np.int64)


@pytest.mark.parametrize("variant", ["auto", "rms_tc"])
def test_is_foreign_full_size(ctx, variant):
    """14,541 entities, 7,991 facts: the whole matrix against the forest walk
    above, and 300 sampled rows against the oracle."""
    n = 14541
    (ci, cx), (ai, ax) = wl.geo_kg(n=n)
    out = torch.zeros((n, wl.words(n)), dtype=torch.int64, device="cuda")
    ctx.is_foreign(dev(wl.csr_to_packed(n, ci, cx).view(np.int64)), dev(wl.csr_to_packed(n, ai, ax).view(np.int64)),
                   n, out, fmt=PACKED, variant=variant)
    got = unpacked(out, n)
    rows = np.random.default_rng(0).choice(n, 300, replace=False).astype(np.int32)
    np.testing.assert_array_equal(got[rows], oracle.is_foreign(n, (ci, cx), (ai, ax), rows=rows))
    want = np.ones((n, n), np.uint8)
    r, c = forest_ipo(n, (ci, cx), (ai, ax))
    want[r, c] = 0
    np.testing.assert_array_equal(got, want)
