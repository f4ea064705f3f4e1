"""Readers for the small text fixtures under tests/golden/ (each cites its passage)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_facts(name):
    """Return (constants list, {predicate: [(a, b), ...]}) from a fixture file."""
    consts = []
    facts = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "constants":
                consts = parts[1:]
            else:
                facts.setdefault(parts[0], []).append(tuple(parts[1:]))
    return consts, facts


def matrix(consts, pairs):
    """Dense 0/1 uint8 matrix of a binary predicate under the constant order."""
    idx = {c: i for i, c in enumerate(consts)}
    m = np.zeros((len(consts), len(consts)), np.uint8)
    for a, b in pairs:
        m[idx[a], idx[b]] = 1
    return m
