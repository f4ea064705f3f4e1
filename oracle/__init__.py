"""CPU oracle for Boolean Matrix Logic Programming closures.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library
never calls it, and it shares no code with the CUDA library: inputs come from
the separate ``workloads`` generators, outputs are plain numpy ``uint8`` 0/1
matrices.

What it computes (paper Sec. 2 Eq. 1, Sec. 3.3 Eq. 4-5, Sec. 3.4 Thm. 1):

* ``closure``      R1+ = sum_{k>=1} R1^k by per-source BFS from successors
* ``reach_rows``   selected rows of R1+ with shortest-path depths
* ``reach_rows_bits`` the same rows as LSB-first uint64 bit rows
* ``smp``          v R1+ for packed source rows (Eq. 5)
* ``seminaive``    semi-naive bottom-up evaluation of p <- base ; p <- rec, p
* ``warshall``     Warshall triple loop (small n)
* ``compose_rows`` rows of (I + R2+) R1 by search
* ``rms_iterations`` number of products the squaring fixpoint issues
* ``alg1_products`` number of products of Algorithm 1 as printed
* ``is_foreign``   rows of the composed program P3 u P4 u P5 of Sec. 3.4

Parity status: every function above is pinned by ``tests/test_oracle_pins.py``
(paper examples, closed forms, invariants, brute force on tiny inputs).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_reach_rows.argtypes = [ctypes.c_int64, _i64p, _i32p, _i32p, ctypes.c_int64, _u8p, _i32p, _i64p]
            lib.oracle_reach_rows_bits.argtypes = [ctypes.c_int64, _i64p, _i32p, _i32p, ctypes.c_int64, _u64p,
                                                   ctypes.c_int64]
            lib.oracle_smp.argtypes = [ctypes.c_int64, _i64p, _i32p, _u64p, ctypes.c_int64, ctypes.c_int64, _u8p, _i32p]
            lib.oracle_seminaive.restype = ctypes.c_int32
            lib.oracle_seminaive.argtypes = [ctypes.c_int64, _u8p, _u8p, _u8p]
            lib.oracle_warshall.argtypes = [ctypes.c_int64, _u8p, _u8p]
            lib.oracle_compose_rows.argtypes = [ctypes.c_int64, _i64p, _i32p, _i64p, _i32p, _i32p, ctypes.c_int64, _u8p]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def set_threads(t: int) -> int:
    """Threads of the oracle's parallel loops (t <= 0 keeps them); returns the previous setting."""
    return int(_L().oracle_set_threads(int(t)))


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr(indptr, indices, n=None):
    ip = np.ascontiguousarray(indptr, np.int64)
    ix = np.ascontiguousarray(indices, np.int32)
    if n is not None:  # the C code trusts its inputs: a row or column index outside [0, n) is refused here
        if len(ip) < n + 1 or (ix.size and (int(ix.min()) < 0 or int(ix.max()) >= n)):
            raise ValueError("CSR does not describe an n = %d relation" % n)
    if ix.size == 0:
        ix = np.zeros(1, np.int32)
    return ip, ix


def reach_rows(n, indptr, indices, sources, want_rows=True):
    """Rows of R1+ for ``sources`` by BFS from successors.

    Returns (rows uint8 [len(sources), n] or None, depth int32, count int64).
    depth[r] is the longest shortest path (>= 1 edge) from sources[r] to any
    node it reaches; count[r] the number of nodes reached.
    """
    ip, ix = _csr(indptr, indices, n)
    src = np.ascontiguousarray(sources, np.int32)
    m = len(src)
    out = np.zeros((m, n), np.uint8) if want_rows else None
    depth = np.zeros(max(m, 1), np.int32)
    count = np.zeros(max(m, 1), np.int64)
    if m and n:
        _L().oracle_reach_rows(n, _p(ip, _i64p), _p(ix, _i32p), _p(src, _i32p), m,
                               _p(out, _u8p) if want_rows else None, _p(depth, _i32p), _p(count, _i64p))
    return out, depth[:m], count[:m]


def reach_rows_bits(n, indptr, indices, sources, ldw=None):
    """Rows of R1+ for ``sources`` as bit rows (uint64 [len(sources), ldw],
    bit j % 64 of word j / 64 least significant first; ldw defaults to
    ceil(n / 64)), by the same BFS as ``reach_rows``."""
    ip, ix = _csr(indptr, indices, n)
    src = np.ascontiguousarray(sources, np.int32)
    ldw = (n + 63) // 64 if ldw is None else int(ldw)
    out = np.zeros((len(src), ldw), np.uint64)
    if len(src) and n:
        _L().oracle_reach_rows_bits(n, _p(ip, _i64p), _p(ix, _i32p), _p(src, _i32p), len(src), _p(out, _u64p), ldw)
    return out


def closure_bits_chunks(n, indptr, indices, rows_per_chunk=4096):
    """R1+ as bit rows, ``rows_per_chunk`` rows at a time: yields (first row, uint64 block)."""
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        yield r0, reach_rows_bits(n, indptr, indices, np.arange(r0, r1, dtype=np.int32))


def closure(n, indptr, indices):
    """Full R1+ (n x n uint8) by per-source BFS."""
    rows, _, _ = reach_rows(n, indptr, indices, np.arange(n, dtype=np.int32))
    return rows if rows is not None else np.zeros((0, 0), np.uint8)


def longest_shortest_path(n, indptr, indices):
    """L = max over pairs in R1+ of the shortest path length (0 if R1+ empty)."""
    _, depth, _ = reach_rows(n, indptr, indices, np.arange(n, dtype=np.int32), want_rows=False)
    return int(depth.max()) if n else 0


def rms_iterations(L: int) -> int:
    """Products issued by the fixpoint R <- R or R.R started from R1.

    After t products R covers every path of length 1..2^t, so R = R1+ once
    2^t >= L, and one more product confirms that nothing changes:
    iterations = ceil(log2 L) + 1, and 1 when L <= 1 (Appendix C Prop. 1
    bounds this by O(log2 n)).
    """
    if L <= 1:
        return 1
    return int(math.ceil(math.log2(L))) + 1


def alg1_products(L0: int) -> int:
    """Products issued by Algorithm 1 as printed: squarings of I + R1 until
    one changes nothing, then the product with R1.

    After t squarings (I + R1)^(2^t) covers the paths of length 0..2^t (the
    diagonal is there from I), so it equals I + R1+ once 2^t >= L0, the
    longest shortest path between two different constants, and one more
    squaring confirms it: ceil(log2 L0) + 1 squarings when L0 >= 2, one when
    L0 <= 1; plus the final product.
    """
    if L0 <= 1:
        return 2
    return int(math.ceil(math.log2(L0))) + 2


def smp(n, indptr, indices, src_rows):
    """v R1+ for each packed (LSB-first uint64) source row; returns (out, levels)."""
    ip, ix = _csr(indptr, indices, n)
    rows = np.ascontiguousarray(src_rows, np.uint64)
    q = rows.shape[0]
    ld = rows.shape[1] if rows.ndim == 2 else 0
    out = np.zeros((q, n), np.uint8)
    lv = np.zeros(max(q, 1), np.int32)
    if q and n:
        _L().oracle_smp(n, _p(ip, _i64p), _p(ix, _i32p), _p(rows, _u64p), q, ld, _p(out, _u8p), _p(lv, _i32p))
    return out, lv[:q]


def seminaive(base, rec=None):
    """Semi-naive evaluation of p <- base ; p <- rec, p on dense 0/1 matrices.

    rec defaults to base (program P2 of Sec. 3.3, giving R1+). Returns
    (P uint8 n x n, rounds).
    """
    b = np.ascontiguousarray(base, np.uint8)
    r = b if rec is None else np.ascontiguousarray(rec, np.uint8)
    n = b.shape[0]
    out = np.zeros((n, n), np.uint8)
    if n == 0:
        return out, 0
    rounds = _L().oracle_seminaive(n, _p(b, _u8p), _p(r, _u8p), _p(out, _u8p))
    return out, int(rounds)


def warshall(m):
    """R1+ by Warshall's triple loop (small n)."""
    a = np.ascontiguousarray(m, np.uint8)
    n = a.shape[0]
    out = np.zeros((n, n), np.uint8)
    if n:
        _L().oracle_warshall(n, _p(a, _u8p), _p(out, _u8p))
    return out


def compose_rows(n, csr1, csr2, rows=None):
    """Rows of P = (I + R2+) R1, the least model of p <- r1 ; p <- r2, p."""
    ip1, ix1 = _csr(*csr1, n)
    ip2, ix2 = _csr(*csr2, n)
    rr = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, np.int32)
    out = np.zeros((len(rr), n), np.uint8)
    if len(rr) and n:
        _L().oracle_compose_rows(n, _p(ip1, _i64p), _p(ix1, _i32p), _p(ip2, _i64p), _p(ix2, _i32p),
                                 _p(rr, _i32p), len(rr), _p(out, _u8p))
    return out


def _dense_to_csr(m):
    r, c = np.nonzero(m)
    ip = np.zeros(m.shape[0] + 1, np.int64)
    np.add.at(ip, r + 1, 1)
    return np.cumsum(ip), c.astype(np.int32)


def is_foreign(n, contains, adjoins, location=None, rows=None):
    """Rows of isForeign for the programs P3, P4, P5 of Sec. 3.4.

    P3: hasPlace = contains+ (per-source BFS). P4: indirectlyPartOf(X,Y) holds
    for adjoins(X,Y), adjoins(Y,X), or hasPlace(Z,X) with
    indirectlyPartOf(Z,Y); its least model is p <- base ; p <- rec, p with
    base = adjoins u adjoins^T and rec(X,Z) = hasPlace(Z,X), evaluated row by
    row by ``compose_rows``. P5: isForeign(X,Y) = location(X), location(Y),
    not indirectlyPartOf(X,Y). contains / adjoins are (indptr, indices);
    location is a 0/1 vector of length n or None (every constant).
    """
    rr = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, np.int32)
    has_place = closure(n, *contains)
    rec = _dense_to_csr(np.ascontiguousarray(has_place.T))
    a = np.zeros((n, n), np.uint8)
    ip, ix = _csr(*adjoins)
    for i in range(n):
        a[i, ix[ip[i]:ip[i + 1]]] = 1
    base = _dense_to_csr(a | a.T)
    ipo = compose_rows(n, base, rec, rr)
    loc = np.ones(n, np.uint8) if location is None else np.asarray(location, np.uint8)
    return (loc[rr][:, None] & loc[None, :] & (1 - ipo)).astype(np.uint8)
