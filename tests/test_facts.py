"""Facts <-> matrices front-end (Sec. 3.2 compilation), host side only."""
import numpy as np
import pytest

import workloads as wl
from golden_io import matrix, read_facts
from paper_2408_10369_gb300 import facts as F

EXAMPLE = """
% Sec. 3.4 example, written as Prolog facts
contains(t1, g2).   contains(g3, t1).
adjoins(g3, g4).
location(g1). location(g2). location(g3). location(g4).
location(t1). location(t2). location(t3).
contains(t1, g2).   % a duplicate is dropped
"""


def test_parse_and_index():
    f = F.parse_facts(EXAMPLE)
    assert f["contains"] == [("t1", "g2"), ("g3", "t1")]
    assert f["adjoins"] == [("g3", "g4")]
    assert len(f["location"]) == 7
    dom = F.Domain.of(f)
    assert dom.names == ["g1", "g2", "g3", "g4", "t1", "t2", "t3"]
    consts, golden = read_facts("p3p5_isforeign.txt")
    np.testing.assert_array_equal(F.relation_matrix(f["contains"], dom), matrix(consts, golden["contains"]))
    v = F.type_vector(f["location"], dom)
    assert int(v[0]) == (1 << 7) - 1


def test_quoting_round_trip():
    f = F.parse_facts("edge('New York', b). edge(b, 'it''s'). edge(b, 'x%y'). edge(3, 4.5). % tail")
    assert f["edge"][0] == ("New York", "b") and f["edge"][2] == ("b", "x%y") and f["edge"][3] == ("3", "4.5")
    dom = F.Domain.of(f)
    m = F.relation_matrix(f["edge"], dom)
    back = F.parse_facts("\n".join(F.matrix_facts("edge", m, dom)))
    assert sorted(back["edge"]) == sorted(f["edge"])


def test_packed_layout_matches_library_layout():
    rng = np.random.default_rng(1)
    m = (rng.random((70, 200)) < 0.2).astype(np.uint8)
    np.testing.assert_array_equal(F.pack(m), wl.pack_rows(m))
    np.testing.assert_array_equal(F.unpack(F.pack(m), 200), m)
    dom = F.Domain(str(i) for i in range(70))
    rows = [(str(i), str(j)) for i, j in zip(*np.nonzero(m[:, :70]))]
    np.testing.assert_array_equal(F.relation_matrix(rows, dom, packed=True), F.pack(m[:, :70]))


@pytest.mark.parametrize("bad", ["path(X, Y) :- edge(X, Y).", "edge(a, b)", "Edge(a, b).", "edge(a, b, c)."])
def test_rejects_non_facts(bad):
    with pytest.raises(ValueError):
        F.parse_facts(bad)
