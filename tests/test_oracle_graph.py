"""Pins of the oracle's 1-skeleton adjacency (every arc at both ends, Sec. 3.5 "Data structure"):
symmetry and arc bookkeeping on random fields, and the closed-form complex of the separable
cosine field (8 minima on a 2x2x2 lattice, 12 1-saddles on its edges, 6 2-saddles on its faces, one
maximum in the middle; every 2-saddle's other arc climbs out through the boundary)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field


def _graph(f):
    e = oracle.compute_all(f, with_minor=False, with_dstar=True)
    return e, oracle.complex_graph(e["counts"], e["lists"], e["min_arcs"], e["max_arcs"], e["dstar"])


def _entries(nodeptr, adj, mult):
    u = np.repeat(np.arange(len(nodeptr) - 1), np.diff(nodeptr))
    return {(int(a), int(b)): int(m) for a, b, m in zip(u, adj, mult)}


@pytest.mark.parametrize("shape,seed", [((5, 4, 6), 1), ((7, 7, 7), 2), ((9, 8, 10), 3)])
def test_symmetry_and_arc_counts(shape, seed):
    e, (nodeptr, adj, mult) = _graph(random_field(shape, seed, "normal"))
    c = [int(x) for x in e["counts"]]
    base = np.cumsum([0] + c)
    d = _entries(nodeptr, adj, mult)
    assert all(d[(b, a)] == m for (a, b), m in d.items())          # both ends
    assert all(a != b for a, b in d)
    for u in range(len(nodeptr) - 1):                              # rows increase
        assert np.all(np.diff(adj[nodeptr[u]:nodeptr[u + 1]].astype(np.int64)) > 0)
    # each 1-saddle: two arcs to minima; each 2-saddle: its arcs that do not leave the domain
    for s in range(c[1]):
        assert sum(m for (a, b), m in d.items() if a == base[1] + s and b < base[1]) == 2
    ma = e["max_arcs"].reshape(-1, 2)
    for t in range(c[2]):
        want = int(np.sum(ma[t] != oracle.NONE))
        assert sum(m for (a, b), m in d.items() if a == base[2] + t and b >= base[3]) == want
    # the saddle-saddle entries are D*
    rows, cols, cnt = e["dstar"]
    for r, col, n in zip(rows, cols, cnt):
        assert d[(int(base[1] + r), int(base[2] + col))] == int(n)
    assert sum(1 for (a, b) in d if base[1] <= a < base[2] and base[2] <= b < base[3]) == len(rows)


def test_cosine_lattice_complex():
    e, (nodeptr, adj, mult) = _graph(fields.cosine_lattice())
    c = [int(x) for x in e["counts"]]
    assert c == [8, 12, 6, 1]
    deg = np.diff(nodeptr)
    assert list(deg[:8]) == [3] * 8                        # a minimum: its 3 lattice edges
    d = _entries(nodeptr, adj, mult)
    for s in range(12):                                    # a 1-saddle: 2 distinct minima
        mins = [(b, m) for (a, b), m in d.items() if a == 8 + s and b < 8]
        assert len(mins) == 2 and all(m == 1 for _, m in mins)
    top = 8 + 12 + 6
    assert sorted(b for (a, b) in d if a == top) == list(range(20, 26))   # the maximum: all 2-saddles
    assert all(d[(top, b)] == 1 for b in range(20, 26))
