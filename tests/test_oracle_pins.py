"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check is a worked example
printed in the paper, a closed form, an invariant of the closure, a library
routine (numpy integer matmul) applied to a plain definition, or brute force
over every digraph on a few nodes.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as wl
from golden_io import matrix, read_facts


def csr(m):
    return wl.csr_from_dense(np.asarray(m))


def bool_mm(a, b):
    """Boolean product via numpy integer matmul (a library primitive)."""
    return ((a.astype(np.int64) @ b.astype(np.int64)) > 0).astype(np.uint8)


def closure_by_powers(m):
    """R+ = R + R^2 + ... + R^n with numpy matmul (paper Sec. 2, Eq. 1 sum)."""
    n = m.shape[0]
    acc = np.zeros_like(m)
    p = m.copy()
    for _ in range(max(n, 1)):
        acc |= p
        p = bool_mm(p, m)
    return acc


def all_three(m):
    n = m.shape[0]
    ip, ix = csr(m)
    a = oracle.closure(n, ip, ix)
    b, _ = oracle.seminaive(m)
    c = oracle.warshall(m)
    return a, b, c


# ------------------------------------------------------- paper examples --
def test_p1_example_printed_output():
    """Sec. 3.2 Example 1 / Appendix B: edge(a,b), edge(b,c) gives path as printed."""
    consts, facts = read_facts("p1_edge_path.txt")
    edge = matrix(consts, facts["edge"])
    want = matrix(consts, facts["path"])
    for got in all_three(edge):
        np.testing.assert_array_equal(got, want)
    assert want.diagonal().sum() == 0  # the printed output is R1+, not I + R1+


def test_p3_p5_isforeign_example():
    """Sec. 3.4: hasPlace = RMS(contains); indirectlyPartOf by composition with
    transposes; isForeign = NEG(indirectlyPartOf): exactly 4 false groundings."""
    consts, facts = read_facts("p3p5_isforeign.txt")
    n = len(consts)
    contains = matrix(consts, facts["contains"])
    adjoins = matrix(consts, facts["adjoins"])
    has_place = oracle.closure(n, *csr(contains))
    # indirectlyPartOf(X,Y) <- adjoins(X,Y) ; adjoins(Y,X) ; hasPlace(Z,X), indirectlyPartOf(Z,Y)
    base = adjoins | adjoins.T
    rec = has_place.T.copy()
    ipo_sn, _ = oracle.seminaive(base, rec)
    ipo_search = oracle.compose_rows(n, csr(base), csr(rec))
    np.testing.assert_array_equal(ipo_sn, ipo_search)
    is_foreign = 1 - ipo_sn  # every constant is a location
    want_false = matrix(consts, facts["not_isForeign"])
    np.testing.assert_array_equal(1 - is_foreign, want_false)
    assert int(is_foreign.sum()) == n * n - 4


def test_is_foreign_oracle_example():
    """The composed-program oracle on the Sec. 3.4 example: 45 of 49 groundings,
    the 4 false ones exactly as listed; a location subset restricts both
    arguments."""
    consts, facts = read_facts("p3p5_isforeign.txt")
    n = len(consts)
    c, a = csr(matrix(consts, facts["contains"])), csr(matrix(consts, facts["adjoins"]))
    got = oracle.is_foreign(n, c, a)
    np.testing.assert_array_equal(1 - got, matrix(consts, facts["not_isForeign"]))
    assert int(got.sum()) == 45
    loc = np.array([1, 1, 1, 1, 0, 0, 0], np.uint8)           # only g1..g4 are locations
    got = oracle.is_foreign(n, c, a, loc)
    assert int(got[4:].sum()) == 0 and int(got[:, 4:].sum()) == 0
    assert int(got.sum()) == 16 - 3                            # (g2, g4), (g3, g4), (g4, g3) stay false
    np.testing.assert_array_equal(oracle.is_foreign(n, c, a, loc, rows=[3, 0]), got[[3, 0]])


def brute_is_foreign(n, contains, adjoins, loc):
    """Naive bottom-up evaluation of P3, P4, P5 over sets of ground atoms."""
    has_place = set(contains)
    while True:
        new = {(x, y) for (x, z) in contains for (z2, y) in has_place if z == z2} - has_place
        if not new:
            break
        has_place |= new
    ipo = set(adjoins) | {(y, x) for (x, y) in adjoins}
    while True:
        new = {(x, y) for (z, x) in has_place for (z2, y) in ipo if z == z2} - ipo
        if not new:
            break
        ipo |= new
    return {(x, y) for x in range(n) for y in range(n) if loc[x] and loc[y] and (x, y) not in ipo}


def test_is_foreign_oracle_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(150):
        n = int(rng.integers(1, 7))
        cm = (rng.random((n, n)) < rng.uniform(0.05, 0.4)).astype(np.uint8)
        am = (rng.random((n, n)) < rng.uniform(0.0, 0.3)).astype(np.uint8)
        loc = (rng.random(n) < 0.7).astype(np.uint8)
        contains = list(zip(*np.nonzero(cm)))
        adjoins = list(zip(*np.nonzero(am)))
        want = np.zeros((n, n), np.uint8)
        for x, y in brute_is_foreign(n, contains, adjoins, loc):
            want[x, y] = 1
        np.testing.assert_array_equal(oracle.is_foreign(n, csr(cm), csr(am), loc), want)


# -------------------------------------------------------- brute force --
def walk_closure(m):
    """(i, j) in R+ iff some walk i -> v1 -> ... -> j of 1..n edges exists,
    enumerated explicitly over all intermediate vertex sequences."""
    n = m.shape[0]
    out = np.zeros_like(m)
    for i in range(n):
        for j in range(n):
            hit = False
            for length in range(1, n + 1):
                for mid in itertools.product(range(n), repeat=length - 1):
                    path = (i,) + mid + (j,)
                    if all(m[path[t], path[t + 1]] for t in range(length)):
                        hit = True
                        break
                if hit:
                    break
            out[i, j] = hit
    return out


def all_digraphs(n):
    for code in range(1 << (n * n)):
        bits = [(code >> b) & 1 for b in range(n * n)]
        yield np.array(bits, np.uint8).reshape(n, n)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_exhaustive_small_walks(n):
    """Every digraph on n <= 3 nodes: the three oracles equal walk enumeration."""
    for m in all_digraphs(n):
        want = walk_closure(m)
        for got in all_three(m):
            np.testing.assert_array_equal(got, want)


def test_exhaustive_n4_bfs_block_diagonal():
    """All 65,536 digraphs on 4 nodes as disjoint blocks of one graph: the BFS
    oracle equals the matrix-power definition block by block."""
    graphs = np.array(list(itertools.product([0, 1], repeat=16)), np.uint8).reshape(-1, 4, 4)
    # matrix-power definition, vectorised over all graphs
    g = graphs.astype(np.int64)
    acc = np.zeros_like(g)
    p = g.copy()
    for _ in range(4):
        acc |= p
        p = (np.einsum("bij,bjk->bik", p, g) > 0).astype(np.int64)
    want = acc.astype(np.uint8)
    per = 1024
    for s in range(0, len(graphs), per):
        blk = graphs[s:s + per]
        k = len(blk)
        n = 4 * k
        src, dst = [], []
        for b in range(k):
            i, j = np.nonzero(blk[b])
            src.append(i + 4 * b)
            dst.append(j + 4 * b)
        ip, ix = wl.csr_from_pairs(n, np.concatenate(src), np.concatenate(dst))
        rows, _, _ = oracle.reach_rows(n, ip, ix, np.arange(n, dtype=np.int32))
        for b in range(k):
            np.testing.assert_array_equal(rows[4 * b:4 * b + 4, 4 * b:4 * b + 4], want[s + b])
            assert rows[4 * b:4 * b + 4].sum() == rows[4 * b:4 * b + 4, 4 * b:4 * b + 4].sum()


def test_random_n4_seminaive_warshall():
    rng = np.random.default_rng(4)
    for _ in range(300):
        m = (rng.random((4, 4)) < 0.35).astype(np.uint8)
        want = closure_by_powers(m)
        b, _ = oracle.seminaive(m)
        np.testing.assert_array_equal(b, want)
        np.testing.assert_array_equal(oracle.warshall(m), want)


# ------------------------------------------------------- closed forms --
@pytest.mark.parametrize("n", [2, 5, 64, 129])
def test_chain_is_strict_upper_triangle(n):
    ip, ix = wl.csr_from_pairs(n, np.arange(n - 1), np.arange(1, n))
    got = oracle.closure(n, ip, ix)
    np.testing.assert_array_equal(got, np.triu(np.ones((n, n), np.uint8), 1))
    assert oracle.longest_shortest_path(n, ip, ix) == n - 1


@pytest.mark.parametrize("n", [1, 2, 7, 100])
def test_cycle_is_all_ones(n):
    ip, ix = wl.csr_from_pairs(n, np.arange(n), (np.arange(n) + 1) % n)
    got = oracle.closure(n, ip, ix)
    np.testing.assert_array_equal(got, np.ones((n, n), np.uint8))
    assert oracle.longest_shortest_path(n, ip, ix) == n  # the way back to i is n edges


def test_complete_digraph_and_empty():
    n = 9
    full = 1 - np.eye(n, dtype=np.uint8)
    for got in all_three(full):
        np.testing.assert_array_equal(got, np.ones((n, n), np.uint8))
    empty = np.zeros((n, n), np.uint8)
    for got in all_three(empty):
        assert got.sum() == 0
    one = np.ones((1, 1), np.uint8)
    for got in all_three(one):
        np.testing.assert_array_equal(got, one)


def test_dag_has_zero_diagonal_and_diag_marks_cycles():
    rng = np.random.default_rng(1)
    n = 60
    dag = np.triu((rng.random((n, n)) < 0.1).astype(np.uint8), 1)
    perm = rng.permutation(n)
    dag = dag[perm][:, perm]
    c = oracle.closure(n, *csr(dag))
    assert c.diagonal().sum() == 0
    # diag(R+)_i = 1 iff i lies on a cycle: add one back edge and check
    m = dag.copy()
    i, j = np.argwhere(c)[0]
    m[j, i] = 1
    c2 = oracle.closure(n, *csr(m))
    on_cycle = np.array([c2[k, k] for k in range(n)])
    want = np.array([bool((c2[i, k] and c2[k, i]) or k in (i, j)) for k in range(n)])
    np.testing.assert_array_equal(on_cycle.astype(bool), want)


def test_symmetric_graph_gives_component_blocks():
    n = 80
    s, d = wl.random_pairs(n, 40, 3)
    m = np.zeros((n, n), np.uint8)
    m[s, d] = 1
    m |= m.T
    c = oracle.closure(n, *csr(m))
    # connected components by union-find
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in zip(*np.nonzero(m)):
        parent[find(a)] = find(b)
    comp = np.array([find(x) for x in range(n)])
    size = np.bincount(comp, minlength=n)
    want = ((comp[:, None] == comp[None, :]) & (size[comp] >= 2)[:, None]).astype(np.uint8)
    np.testing.assert_array_equal(c, want)


# ---------------------------------------------------------- invariants --
@pytest.mark.parametrize("n,d,seed", [(50, 0.8, 0), (120, 1.5, 1), (200, 3.0, 2), (257, 1.0, 3)])
def test_invariants_random_er(n, d, seed):
    ip, ix = wl.er_graph(n, d, seed)
    r = wl.dense_u8(n, ip, ix)
    c = oracle.closure(n, ip, ix)
    assert np.all(c >= r)                                         # R subset of R+
    assert np.all(bool_mm(c, c) <= c)                             # R+ R+ subset of R+
    np.testing.assert_array_equal(oracle.closure(n, *csr(c)), c)  # idempotent
    np.testing.assert_array_equal(c, r | bool_mm(r, c))           # Eq. 1 fixpoint
    np.testing.assert_array_equal(oracle.closure(n, *csr(r.T.copy())), c.T)
    np.testing.assert_array_equal(c, closure_by_powers(r))
    sn, _ = oracle.seminaive(r)
    np.testing.assert_array_equal(sn, c)
    np.testing.assert_array_equal(oracle.warshall(r), c)


def test_resume_from_intermediate():
    """Any R_k with R1 <= R_k <= R1+ has the same closure (restart points)."""
    n = 150
    ip, ix = wl.er_graph(n, 2.0, 7)
    r = wl.dense_u8(n, ip, ix)
    c = oracle.closure(n, ip, ix)
    mid = r | bool_mm(r, r)
    mid = mid | bool_mm(mid, mid)
    np.testing.assert_array_equal(oracle.closure(n, *csr(mid)), c)


# -------------------------------------------------- iteration counts --
def squaring_products(m):
    """Count products of R <- R or R.R (from R1) until one changes nothing."""
    r = m.copy()
    k = 0
    while True:
        k += 1
        nr = r | bool_mm(r, r)
        if np.array_equal(nr, r):
            return k, r
        r = nr


@pytest.mark.parametrize("seed", range(12))
def test_rms_iteration_closed_form(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 70))
    d = float(rng.uniform(0.3, 3.0))
    ip, ix = wl.er_graph(n, d, seed)
    m = wl.dense_u8(n, ip, ix)
    k, fix = squaring_products(m)
    np.testing.assert_array_equal(fix, oracle.closure(n, ip, ix))
    L = oracle.longest_shortest_path(n, ip, ix)
    assert oracle.rms_iterations(L) == k
    assert k <= int(np.ceil(np.log2(max(n, 2)))) + 2  # Appendix C Prop. 1: O(log2 n)


def test_rms_iterations_chain_and_cycle():
    for n in (2, 3, 4, 5, 9, 17, 100):
        ip, ix = wl.csr_from_pairs(n, np.arange(n - 1), np.arange(1, n))
        k, _ = squaring_products(wl.dense_u8(n, ip, ix))
        assert k == oracle.rms_iterations(n - 1)
        ip, ix = wl.csr_from_pairs(n, np.arange(n), (np.arange(n) + 1) % n)
        k, _ = squaring_products(wl.dense_u8(n, ip, ix))
        assert k == oracle.rms_iterations(n)


def offdiag_longest_shortest(m):
    """L0, the longest shortest path between two different constants, by
    Boolean powers: the largest k at which some pair i != j is first reached."""
    n = m.shape[0]
    reach = np.eye(n, dtype=np.uint8)
    p = np.eye(n, dtype=np.uint8)
    L0 = 0
    for k in range(1, n + 1):
        p = bool_mm(p, m)
        if (p & (1 - reach)).any():
            L0 = k
        reach |= p
    return L0


def alg1_literal(m):
    """Algorithm 1 as printed, with numpy matmul: R* = I + R1 squared until a
    squaring changes nothing, then R* R1. Returns (R1+, products)."""
    n = m.shape[0]
    r = m | np.eye(n, dtype=np.uint8)
    k = 0
    while True:
        k += 1
        nr = bool_mm(r, r)
        if np.array_equal(nr, r):
            break
        r = nr
    return bool_mm(r, m), k + 1


@pytest.mark.parametrize("seed", range(12))
def test_alg1_literal_form_matches_closure_and_count(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 70))
    d = float(rng.uniform(0.3, 3.0))
    ip, ix = wl.er_graph(n, d, 100 + seed)
    m = wl.dense_u8(n, ip, ix)
    got, k = alg1_literal(m)
    np.testing.assert_array_equal(got, oracle.closure(n, ip, ix))
    assert k == oracle.alg1_products(offdiag_longest_shortest(m))


def test_alg1_products_chain_and_cycle():
    """A chain or a cycle on n constants has L0 = n - 1."""
    for n in (2, 3, 4, 5, 9, 17, 40):
        for dst in (np.arange(1, n), (np.arange(n) + 1) % n):
            src = np.arange(len(dst))
            m = wl.dense_u8(n, *wl.csr_from_pairs(n, src, dst))
            _, k = alg1_literal(m)
            assert k == oracle.alg1_products(n - 1)


# --------------------------------------------------------------- SMP --
@pytest.mark.parametrize("n,d,q,seed", [(64, 1.2, 5, 0), (200, 2.0, 9, 1), (130, 0.7, 16, 2)])
def test_smp_is_union_of_closure_rows(n, d, q, seed):
    ip, ix = wl.er_graph(n, d, seed)
    r = wl.dense_u8(n, ip, ix)
    c = oracle.warshall(r)
    src = wl.query_rows(n, q, 1, 6, seed)
    v = wl.unpack_rows(src, n)
    got, levels = oracle.smp(n, ip, ix, src)
    np.testing.assert_array_equal(got, bool_mm(v, c))              # Eq. 5: v R1+
    assert np.all(levels <= n)                                      # Prop. 2 bound
    # Algorithm 2 literally: v' = v; v* = v' + v'R until fixpoint; then v* R
    for row in range(q):
        vp = v[row:row + 1].copy()
        while True:
            vs = vp | bool_mm(vp, r)
            if np.array_equal(vs, vp):
                break
            vp = vs
        np.testing.assert_array_equal(got[row:row + 1], bool_mm(vp, r))


# ----------------------------------------------------------- compose --
@pytest.mark.parametrize("n,seed", [(30, 0), (90, 1), (150, 2)])
def test_compose_matches_definition(n, seed):
    ip1, ix1 = wl.er_graph(n, 1.0, seed)
    ip2, ix2 = wl.er_graph(n, 1.5, seed + 100)
    r1 = wl.dense_u8(n, ip1, ix1)
    r2 = wl.dense_u8(n, ip2, ix2)
    want = bool_mm(np.eye(n, dtype=np.uint8) | closure_by_powers(r2), r1)   # (I + R2+) R1
    got = oracle.compose_rows(n, (ip1, ix1), (ip2, ix2))
    np.testing.assert_array_equal(got, want)
    sn, _ = oracle.seminaive(r1, r2)
    np.testing.assert_array_equal(sn, want)
    # with r1 = r2 = R the composition is the closure itself
    np.testing.assert_array_equal(oracle.compose_rows(n, (ip1, ix1), (ip1, ix1)), closure_by_powers(r1))


def test_thread_count_does_not_change_results():
    """The oracle's parallel loops give the same rows on one core as on all."""
    n = 700
    ip, ix = wl.er_graph(n, 1.7, 31)
    many = oracle.closure(n, ip, ix)
    prev = oracle.set_threads(1)
    try:
        one = oracle.closure(n, ip, ix)
        assert oracle.set_threads(0) == 1
    finally:
        oracle.set_threads(prev)
    np.testing.assert_array_equal(one, many)


@pytest.mark.parametrize("n,d,seed", [(1, 0.0, 0), (63, 1.5, 1), (64, 2.0, 2), (200, 1.3, 3), (333, 1.1, 4)])
def test_reach_rows_bits_against_matrix_powers(n, d, seed):
    """The bit-row output, unpacked with numpy (LSB first), is the closure by
    matrix powers; padding bits past n are zero; a wider row stride only adds
    zero words."""
    ip, ix = wl.er_graph(n, d, seed)
    m = wl.dense_u8(n, ip, ix)
    want = closure_by_powers(m)
    bits = oracle.reach_rows_bits(n, ip, ix, np.arange(n, dtype=np.int32))
    assert bits.shape == (n, (n + 63) // 64)
    full = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")
    assert np.array_equal(full[:, :n], want) and not full[:, n:].any()
    wide = oracle.reach_rows_bits(n, ip, ix, np.arange(n, dtype=np.int32), ldw=bits.shape[1] + 2)
    assert np.array_equal(wide[:, :bits.shape[1]], bits) and not wide[:, bits.shape[1]:].any()
    chunks = np.concatenate([blk for _, blk in oracle.closure_bits_chunks(n, ip, ix, rows_per_chunk=50)]) if n else bits
    assert np.array_equal(chunks, bits)
