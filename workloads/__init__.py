"""Seeded synthetic inputs for the Boolean closure workloads.

This package holds no part of the closure method. It draws graphs and query
sets from counter-based SplitMix64 streams (C core in ``gen.c``) and returns
them as numpy arrays: CSR adjacency (``indptr`` int64, ``indices`` int32),
dense 0/1 ``uint8`` matrices, or packed LSB-first ``uint64`` query rows. Both
the CPU oracle and the CUDA path take their inputs from here.

Workload recipes (sizes and distributions follow the paper's experiments in
Sec. 5.1/5.3 and Table 1 and their scaled-up successors):

* ``er_csr``       directed Erdos-Renyi, each ordered pair i != j an edge with
                   probability p (the paper's DG benchmark, Sec. 5.3).
* ``powerlaw_csr`` Zipf out-degrees with preferential-attachment targets.
* ``kg_triples``   knowledge-graph-shaped (head, relation, tail) triples with
                   Zipf relation frequencies (stands in for FB15K-237, Sec. 5.1).
* ``sbm_csr``      stochastic block model.
* ``query_rows``   packed source rows for selective (SMP) queries.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libwlgen.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``_build/libwlgen.so`` with gcc and OpenMP."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.wl_key.restype = ctypes.c_uint64
            lib.wl_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.wl_draw.restype = ctypes.c_uint64
            lib.wl_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.wl_er_count.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, _i64p]
            lib.wl_er_fill.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, _i64p, _i32p]
            lib.wl_powerlaw.restype = ctypes.c_int64
            lib.wl_powerlaw.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _i64p, _i32p]
            lib.wl_query_rows.argtypes = [ctypes.c_int64] * 4 + [ctypes.c_uint64, ctypes.c_int64, _u64p]
            lib.wl_kg_triples.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_uint64, _i32p, _i32p, _i32p]
            lib.wl_sbm_count.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, _i64p]
            lib.wl_sbm_fill.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint64, _i64p, _i32p]
            lib.wl_random_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, _i32p, _i32p]
            lib.wl_sbm_sparse_count.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_uint64, _i64p]
            lib.wl_sbm_sparse_fill.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_uint64, _i64p, _i32p]
            lib.wl_csr_to_packed.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int64, _u64p]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def words(n: int) -> int:
    """uint64 words per packed row of n bits."""
    return (int(n) + 63) // 64


def draw(seed: int, tag: int, counter: int) -> int:
    """One SplitMix64 draw of stream ``tag`` under ``seed`` (for tests)."""
    L = _L()
    return int(L.wl_draw(L.wl_key(seed, tag), counter))


def er_csr(n: int, p: float, seed: int):
    """Directed Erdos-Renyi graph: pair (i, j), i != j, is an edge w.p. p."""
    L = _L()
    cnt = np.zeros(n, np.int64)
    if n > 0:
        L.wl_er_count(n, float(p), seed, _p(cnt, _i64p))
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=indptr[1:])
    indices = np.zeros(max(int(indptr[-1]), 1), np.int32)
    if n > 0:
        L.wl_er_fill(n, float(p), seed, _p(indptr, _i64p), _p(indices, _i32p))
    return indptr, indices[: int(indptr[-1])]


def sbm_csr(n: int, nb: int, p_in: float, p_out: float, seed: int):
    """Stochastic block model with ``nb`` equal blocks."""
    L = _L()
    cnt = np.zeros(n, np.int64)
    L.wl_sbm_count(n, nb, float(p_in), float(p_out), seed, _p(cnt, _i64p))
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=indptr[1:])
    indices = np.zeros(max(int(indptr[-1]), 1), np.int32)
    L.wl_sbm_fill(n, nb, float(p_in), float(p_out), seed, _p(indptr, _i64p), _p(indices, _i32p))
    return indptr, indices[: int(indptr[-1])]


def powerlaw_csr(n: int, alpha: float, kmax: int, seed: int):
    """Zipf(alpha) out-degrees in 1..kmax, preferential-attachment targets."""
    L = _L()
    kcap = max(1, min(kmax, n - 1))
    indptr = np.zeros(n + 1, np.int64)
    indices = np.zeros(max(n * kcap, 1), np.int32)
    nnz = L.wl_powerlaw(n, float(alpha), int(kmax), seed, _p(indptr, _i64p), _p(indices, _i32p))
    return indptr, indices[:nnz].copy()


def query_rows(n: int, q: int, cmin: int, cmax: int, seed: int) -> np.ndarray:
    """q packed source rows (q x words(n) uint64), each with U[cmin, cmax] distinct sources."""
    L = _L()
    ld = words(n)
    rows = np.zeros((q, max(ld, 1)), np.uint64)
    if q > 0 and n > 0:
        L.wl_query_rows(n, q, cmin, cmax, seed, ld, _p(rows, _u64p))
    return rows[:, :ld]


def random_pairs(n: int, m: int, seed: int):
    """m uniform ordered pairs (i, j), i != j."""
    L = _L()
    s = np.zeros(max(m, 1), np.int32)
    d = np.zeros(max(m, 1), np.int32)
    if m > 0:
        L.wl_random_pairs(n, m, seed, _p(s, _i32p), _p(d, _i32p))
    return s[:m], d[:m]


def kg_triples(n_ent: int, n_rel: int, n_triples: int, alpha_r: float, seed: int):
    """Deduplicated (head, relation, tail) triples sorted by (relation, head, tail)."""
    L = _L()
    h = np.zeros(n_triples, np.int32)
    r = np.zeros(n_triples, np.int32)
    t = np.zeros(n_triples, np.int32)
    L.wl_kg_triples(n_ent, n_rel, n_triples, float(alpha_r), seed, _p(h, _i32p), _p(r, _i32p), _p(t, _i32p))
    key = (r.astype(np.int64) * n_ent + h) * n_ent + t
    key = np.unique(key)
    t = (key % n_ent).astype(np.int32)
    h = ((key // n_ent) % n_ent).astype(np.int32)
    r = (key // (n_ent * n_ent)).astype(np.int32)
    return h, r, t


# ------------------------------------------------------------ layouts --
def csr_from_pairs(n: int, src, dst):
    """CSR (sorted, deduplicated) from edge lists."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    key = np.unique(src * n + dst)
    s = key // n
    d = (key % n).astype(np.int32)
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=indptr[1:])
    return indptr, d


def dense_u8(n: int, indptr, indices) -> np.ndarray:
    """Dense n x n uint8 0/1 adjacency from CSR."""
    m = np.zeros((n, n), np.uint8)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    m[rows, np.asarray(indices, np.int64)] = 1
    return m


def csr_from_dense(m: np.ndarray):
    """CSR of a dense 0/1 (any nonzero = 1) square matrix."""
    n = m.shape[0]
    r, c = np.nonzero(m)
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=indptr[1:])
    return indptr, c.astype(np.int32)


def pack_rows(m: np.ndarray) -> np.ndarray:
    """Pack a (rows x n) 0/1 matrix to LSB-first uint64 words per row."""
    rows, n = m.shape
    ld = words(n)
    b = np.packbits((np.asarray(m) != 0).astype(np.uint8), axis=1, bitorder="little")
    out = np.zeros((rows, ld * 8), np.uint8)
    out[:, : b.shape[1]] = b
    return out.view(np.uint64).reshape(rows, ld)


def unpack_rows(p: np.ndarray, n: int) -> np.ndarray:
    """Inverse of ``pack_rows``: (rows x words) uint64 -> (rows x n) uint8."""
    p = np.ascontiguousarray(p, dtype=np.uint64)
    b = np.unpackbits(p.view(np.uint8).reshape(p.shape[0], -1), axis=1, bitorder="little")
    return b[:, :n].astype(np.uint8)


# ------------------------------------------------------------ recipes --
def er_graph(n: int, mean_degree: float, seed: int):
    """ER graph with p = mean_degree / (n - 1)."""
    p = 0.0 if n <= 1 else float(mean_degree) / (n - 1)
    return er_csr(n, p, seed)


def kg_relations(n_ent=15000, n_rel=1345, n_triples=483000, alpha_r=1.1, seed=0):
    """Per-relation local problems of the KG workload.

    Returns a list of dicts {rel, n, entities, indptr, indices}: the relation's
    active entities (sorted union of heads and tails, mapped to 0..n-1 in
    order) and its local CSR adjacency.
    """
    h, r, t = kg_triples(n_ent, n_rel, n_triples, alpha_r, seed)
    out = []
    bounds = np.searchsorted(r, np.arange(n_rel + 1))
    for rel in range(n_rel):
        a, b = bounds[rel], bounds[rel + 1]
        if b <= a:
            continue
        hh, tt = h[a:b], t[a:b]
        ents = np.unique(np.concatenate([hh, tt]))
        lh = np.searchsorted(ents, hh)
        lt = np.searchsorted(ents, tt)
        indptr, indices = csr_from_pairs(len(ents), lh, lt)
        out.append(dict(rel=rel, n=len(ents), entities=ents, indptr=indptr, indices=indices))
    return out


def kg_compose_pairs(rels, count=200, seed=0):
    """``count`` seeded (r1, r2) index pairs into ``rels`` with r1 != r2."""
    L = _L()
    key = L.wl_key(seed, 12)
    m = len(rels)
    pairs = []
    c = 0
    while len(pairs) < count and m > 1:
        a = int(L.wl_draw(key, c) % m)
        b = int(L.wl_draw(key, c + 1) % m)
        c += 2
        if a != b:
            pairs.append((a, b))
    return pairs


def union_space(rel1, rel2):
    """Map two relations onto the sorted union of their active entities."""
    ents = np.union1d(rel1["entities"], rel2["entities"])
    n = len(ents)

    def remap(rel):
        rows = np.repeat(np.arange(rel["n"]), np.diff(rel["indptr"]))
        s = np.searchsorted(ents, rel["entities"][rows])
        d = np.searchsorted(ents, rel["entities"][rel["indices"]])
        return csr_from_pairs(n, s, d)

    return n, ents, remap(rel1), remap(rel2)


# ------------------------------------------------------- mixed corpus --
def sbm_sparse_csr(n: int, nb: int, p_in: float, p_out: float, seed: int):
    """Sparse SBM (nb = 1: ER) by geometric skip sampling, O(n + m)."""
    L = _L()
    cnt = np.zeros(max(n, 1), np.int64)
    if n > 0:
        L.wl_sbm_sparse_count(n, nb, float(p_in), float(p_out), seed, _p(cnt, _i64p))
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(cnt[:n], out=indptr[1:])
    indices = np.zeros(max(int(indptr[-1]), 1), np.int32)
    if n > 0:
        L.wl_sbm_sparse_fill(n, nb, float(p_in), float(p_out), seed, _p(indptr, _i64p), _p(indices, _i32p))
    return indptr, indices[: int(indptr[-1])]


def csr_to_packed(n: int, indptr, indices) -> np.ndarray:
    """Packed LSB-first rows (n x words(n) uint64) straight from CSR."""
    ld = words(n)
    rows = np.zeros((max(n, 1), max(ld, 1)), np.uint64)
    ip = np.ascontiguousarray(indptr, np.int64)
    ix = np.ascontiguousarray(indices, np.int32)
    if ix.size == 0:
        ix = np.zeros(1, np.int32)
    if n > 0:
        _L().wl_csr_to_packed(n, _p(ip, _i64p), _p(ix, _i32p), ld, _p(rows, _u64p))
    return rows[:n, :ld]


def geo_kg(n: int = 14541, n_contains: int = 5993, n_adjoins: int = 1998, n_roots: int = 200, seed: int = 0):
    """A place hierarchy with neighbours, the shape of the location subset of
    FB15K-237 used for isForeign (14,541 entities, 7,991 facts).

    contains(p, c): entities are put in a random order; the first n_roots are
    top-level regions, each of the next n_contains entities gets one parent
    among the entities before it, drawn from an urn holding every earlier
    entity once plus one copy per child it already has (preferential
    attachment, so a few regions contain many places). The hierarchy is a
    forest, hence acyclic. adjoins(a, b): n_adjoins uniform pairs a != b,
    deduplicated. Returns (contains CSR, adjoins CSR).
    """
    order = sorted(range(n), key=lambda i: draw(seed, 40, i))
    urn = list(order[:n_roots])
    src, dst = [], []
    for t in range(n_roots, min(n, n_roots + n_contains)):
        child = order[t]
        parent = urn[draw(seed, 41, t) % len(urn)]
        src.append(parent)
        dst.append(child)
        urn.append(child)
        urn.append(parent)
    contains = csr_from_pairs(n, np.array(src, np.int64), np.array(dst, np.int64))
    a, b = random_pairs(n, n_adjoins, wl_seed(seed, 42))
    return contains, csr_from_pairs(n, a, b)


def wl_seed(seed: int, tag: int) -> int:
    """A derived 63-bit seed for a sub-stream."""
    return draw(seed, tag, 0) >> 1


FAMILIES = ("er", "powerlaw", "chain_grid", "sbm")


def _unit(seed, tag, c):
    return (draw(seed, tag, c) >> 11) * (1.0 / 9007199254740992.0)


def corpus_graph(index: int, n_min: int = 256, n_max: int = 32768):
    """Graph `index` of the mixed corpus (seed = index).

    n is log-uniform in [n_min, n_max]; the family is uniform over ER (mean
    out-degree U[0.5, 8]), power law (alpha U[1.8, 3], degrees <= 1000),
    chain or 2-D grid (right/down edges) plus round(1 % of n) random
    shortcuts, and an 8-block SBM (mean out-degree U[0.5, 8], in:out
    probability ratio U[4, 32]). Returns a dict with n, family, params, CSR.
    """
    s = 1_000_003 + int(index)
    fam = FAMILIES[draw(s, 20, 0) % 4]
    u = _unit(s, 20, 1)
    n = int(round(n_min * (n_max / n_min) ** u))
    n = max(n_min, min(n_max, n))
    params = {}
    if fam == "er":
        d = 0.5 + 7.5 * _unit(s, 20, 2)
        params["mean_degree"] = d
        ip, ix = sbm_sparse_csr(n, 1, d / (n - 1), d / (n - 1), s)
    elif fam == "powerlaw":
        a = 1.8 + 1.2 * _unit(s, 20, 2)
        params["alpha"] = a
        ip, ix = powerlaw_csr(n, a, 1000, s)
    elif fam == "chain_grid":
        grid = draw(s, 20, 2) % 2 == 1
        params["shape"] = "grid" if grid else "chain"
        if grid:
            side = max(2, int(np.sqrt(n)))
            idx = np.arange(n)
            r, c = idx // side, idx % side
            right = idx[(c + 1 < side) & (idx + 1 < n)]
            down = idx[idx + side < n]
            src = np.concatenate([right, down])
            dst = np.concatenate([right + 1, down + side])
        else:
            src = np.arange(n - 1)
            dst = src + 1
        m = max(1, int(round(0.01 * n)))
        a, b = random_pairs(n, m, s)
        ip, ix = csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([dst, b]))
    else:
        d = 0.5 + 7.5 * _unit(s, 20, 2)
        ratio = 4.0 + 28.0 * _unit(s, 20, 3)
        B = n / 8.0
        p_out = d / (ratio * (B - 1) + (n - B))
        params.update(mean_degree=d, ratio=ratio)
        ip, ix = sbm_sparse_csr(n, 8, min(1.0, ratio * p_out), p_out, s)
    return dict(index=int(index), family=fam, n=n, params=params, indptr=ip, indices=ix)
