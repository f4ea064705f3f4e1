"""Grouped batch (one persistent launch per iteration, device loop in a CUDA
graph) and the single-problem device loop: bit-exact against the oracle."""
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


def kg_problem_set(n_ent, n_rel, n_triples, n_pairs, seed, fmt):
    rels = wl.kg_relations(n_ent=n_ent, n_rel=n_rel, n_triples=n_triples, seed=seed)
    items, expect, keep = [], [], []
    for r in rels:
        n = r["n"]
        m = wl.dense_u8(n, r["indptr"], r["indices"])
        R = dev(m if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(m).view(np.int64))
        out = torch.zeros_like(R)
        keep += [R, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=fmt))
        expect.append(("closure", n, r["indptr"], r["indices"]))
    for a, b in wl.kg_compose_pairs(rels, n_pairs, seed):
        n, ents, c1, c2 = wl.union_space(rels[a], rels[b])
        m1, m2 = wl.dense_u8(n, *c1), wl.dense_u8(n, *c2)
        if fmt != bmlp.BMLP_FMT_U8:
            m1, m2 = wl.pack_rows(m1).view(np.int64), wl.pack_rows(m2).view(np.int64)
        R1, R2 = dev(m1), dev(m2)
        out = torch.zeros_like(R1)
        keep += [R1, R2, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=n, R1=R1, R2=R2, out=out, fmt=fmt))
        expect.append(("compose", n, c1, c2))
    return items, expect, keep


def check(items, expect, iters=None):
    for it, ex in zip(items, expect):
        got = it["out"].cpu().numpy()
        n = ex[1]
        if it["fmt"] == bmlp.BMLP_FMT_PACKED64:
            got = wl.unpack_rows(got.view(np.uint64), n)
        if ex[0] == "closure":
            want = oracle.closure(n, ex[2], ex[3])
        else:
            want = oracle.compose_rows(n, ex[2], ex[3])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("variant", ["auto", "rms_tc", "rms_packed"])
@pytest.mark.parametrize("fmt", [bmlp.BMLP_FMT_U8, bmlp.BMLP_FMT_PACKED64])
def test_batch_kg_small(ctx, variant, fmt):
    items, expect, keep = kg_problem_set(1500, 40, 9000, 8, 3, fmt)
    iters = ctx.batch_run(items, variant=variant)
    torch.cuda.synchronize()
    check(items, expect)
    # closure iteration counts follow the closed form
    for it, ex, k in zip(items, expect, iters):
        if ex[0] == "closure":
            assert k == oracle.rms_iterations(oracle.longest_shortest_path(ex[1], ex[2], ex[3]))


def test_batch_repeat_uses_cached_graph(ctx):
    items, expect, keep = kg_problem_set(800, 20, 4000, 4, 5, bmlp.BMLP_FMT_U8)
    a = ctx.batch_run(items)
    for it in items:
        it["out"].zero_()
    b = ctx.batch_run(items)
    torch.cuda.synchronize()
    assert a == b
    check(items, expect)


def test_batch_autotune_then_run(ctx, tmp_path):
    items, expect, keep = kg_problem_set(1200, 30, 7000, 0, 7, bmlp.BMLP_FMT_U8)
    cache = str(tmp_path / "tune.txt")
    ctx.batch_autotune(items, cache)
    with open(cache) as f:
        lines = f.read().strip().splitlines()
    assert lines and all(len(ln.split()) == 5 for ln in lines)
    ctx.batch_autotune(items, cache)        # second call reads the cache
    ctx.batch_run(items)
    torch.cuda.synchronize()
    check(items, expect)


def test_batch_edge_cases(ctx):
    n = 5
    R = dev(np.roll(np.eye(n, dtype=np.uint8), 1, axis=1))
    out = torch.zeros_like(R)
    E = torch.zeros((1, 1), dtype=torch.uint8, device="cuda")
    items = [dict(n=0, R1=None, out=None), dict(n=n, R1=R, out=out, reflexive=True),
             dict(n=1, R1=E, out=torch.zeros_like(E))]
    iters = ctx.batch_run(items)
    torch.cuda.synchronize()
    assert iters[0] == 0
    np.testing.assert_array_equal(out.cpu().numpy(), np.ones((n, n), np.uint8))
    assert items[2]["out"].item() == 0


@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed"])
@pytest.mark.parametrize("n,d,seed", [(1, 0.0, 0), (65, 1.5, 1), (300, 1.2, 2), (1000, 2.0, 3), (2000, 1.0, 4)])
def test_single_problem_device_loop(ctx, variant, n, d, seed):
    ip, ix = wl.er_graph(n, d, seed)
    R = dev(wl.dense_u8(n, ip, ix))
    out = torch.zeros_like(R)
    it = ctx.rms(R, n, out, variant=variant, loop=bmlp.BMLP_LOOP_GRAPH)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.closure(n, ip, ix))
    assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))


@pytest.mark.parametrize("fmt", [bmlp.BMLP_FMT_U8, bmlp.BMLP_FMT_PACKED64])
def test_batch_mixes_solo_and_grouped_problems(ctx, fmt):
    """Problems with n >= 4096 run as device-driven single-problem pipelines
    (bit rows, then 4-bit operands) inside the batch graph, the others in the
    grouped batch; every output and every iteration count as for the problem
    alone."""
    items, expect, keep = [], [], []
    for n, d, seed in [(8300, 2.0, 1), (300, 1.5, 2), (8250, 0.7, 3), (900, 1.2, 4)]:
        ip, ix = wl.er_graph(n, d, seed)
        m = wl.dense_u8(n, ip, ix)
        R = dev(m if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(m).view(np.int64))
        out = torch.zeros_like(R)
        keep += [R, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=fmt))
        expect.append(("closure", n, ip, ix))
    n = 8400
    c1, c2 = wl.er_graph(n, 1.0, 5), wl.er_graph(n, 1.1, 6)
    m1, m2 = wl.dense_u8(n, *c1), wl.dense_u8(n, *c2)
    if fmt != bmlp.BMLP_FMT_U8:
        m1, m2 = wl.pack_rows(m1).view(np.int64), wl.pack_rows(m2).view(np.int64)
    R1, R2 = dev(m1), dev(m2)
    out = torch.zeros_like(R1)
    keep += [R1, R2, out]
    items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=n, R1=R1, R2=R2, out=out, fmt=fmt))
    expect.append(("compose", n, c1, c2))
    iters = ctx.batch_run(ctx.problems(items), variant="rms_tc")
    torch.cuda.synchronize()
    check(items, expect)
    for k in range(4):
        _, n, ip, ix = expect[k]
        assert iters[k] == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    # one graph launch: the host waits once, for the results
    assert ctx.stats()["host_syncs"] == 1


@pytest.mark.parametrize("fmt", [bmlp.BMLP_FMT_U8, bmlp.BMLP_FMT_PACKED64])
def test_batch_of_large_problems_only(ctx, fmt):
    """Only problems with n >= 4096 (no grouped part): a path-like relation
    (many squarings on bit rows before the tensor cores take over), a sparse
    one that finishes on bit rows, a dense one that goes straight to the
    tensor cores, a reflexive closure and a composition, all in one graph."""
    items, expect, keep = [], [], []
    cases = [("chain", 5000, 0.01, 11), ("er", 4100, 0.6, 12), ("er", 4500, 6.0, 13), ("refl", 4200, 1.3, 14)]
    for kind, n, p, seed in cases:
        if kind == "chain":
            src = np.arange(n - 1)
            dst = src + 1
            a, b = wl.random_pairs(n, int(p * n), seed)
            ip, ix = wl.csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([dst, b]))
        else:
            ip, ix = wl.er_graph(n, p, seed)
        m = wl.dense_u8(n, ip, ix)
        R = dev(m if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(m).view(np.int64))
        out = torch.zeros_like(R)
        keep += [R, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=fmt, reflexive=kind == "refl"))
        expect.append((kind, n, ip, ix))
    nc = 4300
    c1, c2 = wl.er_graph(nc, 1.2, 15), wl.er_graph(nc, 0.9, 16)
    m1, m2 = wl.dense_u8(nc, *c1), wl.dense_u8(nc, *c2)
    if fmt != bmlp.BMLP_FMT_U8:
        m1, m2 = wl.pack_rows(m1).view(np.int64), wl.pack_rows(m2).view(np.int64)
    R1, R2 = dev(m1), dev(m2)
    out = torch.zeros_like(R1)
    keep += [R1, R2, out]
    items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=nc, R1=R1, R2=R2, out=out, fmt=fmt))
    iters = ctx.batch_run(items)
    torch.cuda.synchronize()
    assert ctx.stats()["host_syncs"] == 1
    for it, (kind, n, ip, ix), k in zip(items, expect, iters):
        got = it["out"].cpu().numpy()
        if fmt == bmlp.BMLP_FMT_PACKED64:
            got = wl.unpack_rows(got.view(np.uint64), n)
        want = oracle.closure(n, ip, ix)
        if kind == "refl":
            want = want | np.eye(n, dtype=np.uint8)
        np.testing.assert_array_equal(got, want)
        assert k == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    got = items[-1]["out"].cpu().numpy()
    if fmt == bmlp.BMLP_FMT_PACKED64:
        got = wl.unpack_rows(got.view(np.uint64), nc)
    np.testing.assert_array_equal(got, oracle.compose_rows(nc, c1, c2))
    # the same problems again reuse the cached graph
    for it in items:
        it["out"].zero_()
    assert ctx.batch_run(items) == iters


def test_single_problem_device_loop_large(ctx):
    """loop = BMLP_LOOP_GRAPH with n >= 4096: the device-driven pipeline
    (bit rows, then 4-bit tensor-core squarings) as a batch of one."""
    n = 6000
    ip, ix = wl.er_graph(n, 1.7, 21)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros_like(P)
    it = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_tc", loop=bmlp.BMLP_LOOP_GRAPH)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), oracle.closure(n, ip, ix))
    assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    assert ctx.stats()["host_syncs"] == 1


@pytest.mark.parametrize("fmt", [bmlp.BMLP_FMT_U8, bmlp.BMLP_FMT_PACKED64])
def test_batch_frontier_engine(ctx, fmt):
    """Closures with variant smp_packed in a batch: every row of each is one
    query of one grouped frontier launch, next to squaring problems and a
    composition; every output bit and the level counts (deepest BFS level + 1)
    against the oracle."""
    items, expect, keep = [], [], []
    cases = [(1, 0.0, 1, "smp_packed"), (64, 1.5, 2, "smp_packed"), (700, 1.2, 3, "smp_packed"),
             (1500, 2.5, 4, "rms_tc"), (2100, 0.9, 5, "smp_packed"), (333, 3.0, 6, "rms_packed"),
             (4000, 1.1, 7, "smp_packed")]
    for n, d, seed, v in cases:
        ip, ix = wl.er_graph(n, d, seed)
        m = wl.dense_u8(n, ip, ix)
        R = dev(m if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(m).view(np.int64))
        out = torch.zeros_like(R)
        keep += [R, out]
        items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=fmt, variant=v))
        expect.append(("closure", n, ip, ix))
    n = 900
    c1, c2 = wl.er_graph(n, 1.0, 8), wl.er_graph(n, 1.3, 9)
    m1, m2 = wl.dense_u8(n, *c1), wl.dense_u8(n, *c2)
    if fmt != bmlp.BMLP_FMT_U8:
        m1, m2 = wl.pack_rows(m1).view(np.int64), wl.pack_rows(m2).view(np.int64)
    R1, R2 = dev(m1), dev(m2)
    out = torch.zeros_like(R1)
    keep += [R1, R2, out]
    items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=n, R1=R1, R2=R2, out=out, fmt=fmt))
    expect.append(("compose", n, c1, c2))
    iters = ctx.batch_run(items)
    torch.cuda.synchronize()
    check(items, expect)
    for (n, d, seed, v), ex, k in zip(cases, expect, iters):
        ip, ix = ex[2], ex[3]
        if v == "smp_packed":
            _, depth, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32), want_rows=False)
            assert k == int(depth.max()) + 1, (n, k)
        else:
            assert k == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    # the whole batch with the frontier engine, and again from the cached graph
    for it in items:
        it["out"].zero_()
        it.pop("variant", None)
    ctx.batch_run(items, variant="smp_packed")
    ctx.batch_run(items, variant="smp_packed")
    torch.cuda.synchronize()
    check(items, expect)


def chain_tail_graph(n0=9000, tail=60, seed=33):
    """A dense random part with a chain of `tail` nodes hanging off it: the chain's columns are reached by most
    rows only after several squarings, so the squarings restricted to the rows and columns holding zeros find new
    ones before the closure is reached."""
    n = n0 + tail
    ip0, ix0 = wl.er_graph(n0, 5.0, seed)
    src = np.concatenate([np.repeat(np.arange(n0), np.diff(ip0)), [0], n0 + np.arange(tail - 1)])
    dst = np.concatenate([ix0, [n0], n0 + 1 + np.arange(tail - 1)])
    ip, ix = wl.csr_from_pairs(n, src, dst)
    return n, ip, ix


@pytest.mark.parametrize("fmt", [bmlp.BMLP_FMT_U8, bmlp.BMLP_FMT_PACKED64])
def test_device_pipeline_restricted_squaring(ctx, fmt):
    """Large closures whose last squarings run only on the rows and columns holding zeros, inside the batch graph
    (IF nodes in the tensor-core loop of the device-driven pipeline): a dense ER closure (only the confirming
    squaring is restricted), the chain-tail graph (restricted squarings that find new ones), a composition whose
    R2 is that graph, and a small closure beside them; every bit against the oracle, and each closure's count of
    squarings is Algorithm 1's."""
    specs = []
    n, ip, ix = 12000, *wl.er_graph(12000, 4.0, 31)
    specs.append(("closure", n, ip, ix))
    specs.append(("closure", *chain_tail_graph()))
    n2, ip2, ix2 = chain_tail_graph()
    ip1, ix1 = wl.er_graph(n2, 2.0, 35)
    specs.append(("compose", n2, (ip1, ix1), (ip2, ix2)))
    specs.append(("closure", 700, *wl.er_graph(700, 2.0, 36)))
    items, expect, keep = [], [], []
    for sp in specs:
        if sp[0] == "closure":
            _, n, ip, ix = sp
            m = wl.dense_u8(n, ip, ix)
            R = dev(m if fmt == bmlp.BMLP_FMT_U8 else wl.pack_rows(m).view(np.int64))
            out = torch.zeros_like(R)
            keep += [R, out]
            items.append(dict(kind=bmlp.BMLP_PROBLEM_CLOSURE, n=n, R1=R, out=out, fmt=fmt))
            expect.append(("closure", n, ip, ix))
        else:
            _, n, c1, c2 = sp
            m1, m2 = wl.dense_u8(n, *c1), wl.dense_u8(n, *c2)
            if fmt != bmlp.BMLP_FMT_U8:
                m1, m2 = wl.pack_rows(m1).view(np.int64), wl.pack_rows(m2).view(np.int64)
            R1, R2 = dev(m1), dev(m2)
            out = torch.zeros_like(R1)
            keep += [R1, R2, out]
            items.append(dict(kind=bmlp.BMLP_PROBLEM_COMPOSE, n=n, R1=R1, R2=R2, out=out, fmt=fmt))
            expect.append(("compose", n, c1, c2))
    iters = ctx.batch_run(items, variant="rms_tc")
    torch.cuda.synchronize()
    check(items, expect)
    for it, ex in zip(iters, expect):
        if ex[0] == "closure":
            assert it == oracle.rms_iterations(oracle.longest_shortest_path(ex[1], ex[2], ex[3]))
