"""Datalog facts <-> Boolean matrices (the compilation step of paper Sec. 3.2).

A set of ground facts over a finite set of constants becomes one n x n
Boolean matrix per dyadic predicate: constant c gets index i(c), and
p(a, b) holds iff P[i(a)][i(b)] = 1 (Sec. 3.2); a monadic (type) predicate
becomes a bit vector. Results of the GPU algorithms are turned back into
facts the same way. This module is host-side I/O only: parsing, the constant
index, and array layout; every closure, composition and operator runs in the
CUDA library.

Accepted syntax: one fact per clause, ``name(arg)`` or ``name(arg1, arg2)``
terminated by ``.``; arguments are Prolog atoms (lower-case identifiers),
numbers, or quoted atoms; ``%`` starts a comment. Rules are not parsed: the
programs themselves are the calls of the library (bmlp_rms, bmlp_compose,
bmlp_is_foreign, ...).
"""
from __future__ import annotations

import re

import numpy as np

_ATOM = r"(?:'(?:[^'\\]|\\.|'')*'|[a-z][A-Za-z0-9_]*|-?\d+(?:\.\d+)?)"
_FACT = re.compile(r"\s*([a-z][A-Za-z0-9_]*)\s*\(\s*(" + _ATOM + r")\s*(?:,\s*(" + _ATOM + r")\s*)?\)\s*\.")


def _unquote(a: str) -> str:
    """Quoted atom -> its text ('' and backslash escapes)."""
    if len(a) >= 2 and a[0] == "'" and a[-1] == "'":
        return re.sub(r"\\(.)|''", lambda m: m.group(1) if m.group(1) is not None else "'", a[1:-1])
    return a


def parse_facts(text: str):
    """{predicate: [tuple of constants, ...]} in order of appearance
    (duplicates removed). Raises ValueError on anything that is not a fact."""
    out: dict[str, list[tuple[str, ...]]] = {}
    seen: set[tuple] = set()
    body = text
    pos = 0
    while True:
        while pos < len(body) and (body[pos].isspace() or body[pos] == "%"):
            if body[pos] == "%":  # comment to the end of the line
                nl = body.find("\n", pos)
                pos = len(body) if nl < 0 else nl
            else:
                pos += 1
        if pos >= len(body):
            break
        m = _FACT.match(body, pos)
        if not m:
            raise ValueError("not a ground fact near: %r" % body[pos:pos + 40])
        name, a, b = m.group(1), _unquote(m.group(2)), m.group(3)
        args = (a,) if b is None else (a, _unquote(b))
        key = (name, args)
        if key not in seen:
            seen.add(key)
            out.setdefault(name, []).append(args)
        pos = m.end()
    return out


class Domain:
    """The constant index of Sec. 3.2: a bijection between constants and 0..n-1."""

    def __init__(self, constants=()):
        self.names: list[str] = []
        self.index: dict[str, int] = {}
        for c in constants:
            self.add(c)

    @classmethod
    def of(cls, facts: dict, predicates=None, sort=True):
        """The constants appearing in the given predicates (all by default)."""
        cs = set()
        for p, rows in facts.items():
            if predicates is None or p in predicates:
                for r in rows:
                    cs.update(r)
        return cls(sorted(cs) if sort else cs)

    def add(self, c: str) -> int:
        if c not in self.index:
            self.index[c] = len(self.names)
            self.names.append(c)
        return self.index[c]

    def __len__(self):
        return len(self.names)

    def pairs(self, rows) -> np.ndarray:
        """m x 2 int32 indices of binary facts (every constant must be known)."""
        a = np.array([[self.index[x], self.index[y]] for x, y in rows], np.int32)
        return a.reshape(-1, 2)


def relation_matrix(rows, dom: Domain, packed: bool = False) -> np.ndarray:
    """n x n uint8 0/1 matrix of binary facts, or packed rows (n x ceil(n/64)
    uint64, bit j of row i at bit j % 64 of word j / 64)."""
    n = len(dom)
    m = np.zeros((n, n), np.uint8)
    p = dom.pairs(rows)
    if len(p):
        m[p[:, 0], p[:, 1]] = 1
    return pack(m) if packed else m


def type_vector(rows, dom: Domain) -> np.ndarray:
    """Packed bit vector (ceil(n/64) uint64) of a monadic predicate."""
    n = len(dom)
    v = np.zeros((1, n), np.uint8)
    for (x,) in rows:
        v[0, dom.index[x]] = 1
    return pack(v)[0]


def pack(m: np.ndarray) -> np.ndarray:
    """0/1 rows -> packed LSB-first uint64 words."""
    rows, n = m.shape
    ld = (n + 63) // 64
    bits = np.zeros((rows, ld * 64), np.uint8)
    bits[:, :n] = m != 0
    return np.packbits(bits, axis=1, bitorder="little").view("<u8").reshape(rows, ld)


def unpack(p: np.ndarray, n: int) -> np.ndarray:
    """Packed LSB-first uint64 rows -> 0/1 uint8 rows of length n."""
    rows = p.shape[0]
    b = np.unpackbits(np.ascontiguousarray(p).view(np.uint8).reshape(rows, -1), axis=1, bitorder="little")
    return b[:, :n].astype(np.uint8)


def matrix_facts(name: str, m: np.ndarray, dom: Domain, packed: bool = False):
    """The facts name(a, b) of a result matrix (u8 or packed), row-major order."""
    if packed:
        m = unpack(m, len(dom))
    r, c = np.nonzero(m)
    return ["%s(%s, %s)." % (name, _quote(dom.names[i]), _quote(dom.names[j])) for i, j in zip(r, c)]


def _quote(a: str) -> str:
    if re.fullmatch(r"[a-z][A-Za-z0-9_]*|-?\d+(?:\.\d+)?", a):
        return a
    return "'" + a.replace("\\", "\\\\").replace("'", "''") + "'"
