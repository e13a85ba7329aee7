"""Pins for the CPU oracle: checks against what the mathematics fixes, not against itself.

* Euler characteristic of a box: #min - #1s + #2s - #max = 1 (every field).
* Structural invariants of a discrete gradient (Sec. 2.2): each cell in at most one pair,
  pairs are facet/cofacet, no non-trivial closed V-path (acyclic modified Hasse diagram),
  both cells of a pair share their maximal vertex (lower-star locality).
* Closed form for the 0-1 pairs: a non-minimal vertex is paired with the edge to its
  lowest lower neighbour; a vertex is critical iff no axis neighbour is lower.
* Lower-star persistent homology by textbook Z2 column reduction: the number of critical
  k-cells equals the number of k-cells that open or close a homology class of non-zero
  persistence, plus essential classes (Robins, Wood, Sheppard 2011).
* Analytic fields with known critical counts (bowl, linear, inverted bowl, cosine lattice).
* Saddle-saddle path counts against exhaustive enumeration of V-paths downward from every
  2-saddle (independent of the oracle's upward DAG walk), and against the paper's own
  iterated-product formulation (Sec. 3.3) in exact Python integers.
* Destination minima against steepest descent on the raw field.
* Cells of the saddle-saddle arcs of multiplicity 1 against the same downward V-path
  enumeration: exactly one path, cell for cell.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import Complex, pairs_dict, random_field, vertex_rank

NONE = 0xFFFFFFFF

SMALL_SHAPES = [(2, 2, 2), (2, 3, 4), (3, 3, 3), (4, 3, 2), (4, 4, 4), (5, 4, 3), (3, 5, 5)]


def _dims(f):
    nz, ny, nx = f.shape
    return (nx, ny, nz)


def _fields_small():
    out = []
    for i, shp in enumerate(SMALL_SHAPES):
        out.append(random_field(shp, 10 + i, "normal"))
        out.append(random_field(shp, 50 + i, "ties"))
    return out


# ----------------------------------------------------------------------------------
# helpers written from the definitions
# ----------------------------------------------------------------------------------
def persistence_critical_counts(f):
    """Critical-cell counts implied by lower-star persistent homology (Z2 column reduction)."""
    C = Complex(_dims(f))
    rank = vertex_rank(f)
    val = {c: max(rank[v] for v in C.vertices(c)) for c in C.cells()}
    order = sorted(C.cells(), key=lambda c: (val[c], C.dim(c), c))
    pos = {c: i for i, c in enumerate(order)}
    low_owner = {}
    cols = []
    paired = set()
    counts = [0, 0, 0, 0]
    for j, c in enumerate(order):
        col = {pos[x] for x in C.facets(c)}
        while col:
            low = max(col)
            if low not in low_owner:
                break
            col ^= cols[low_owner[low]]
        cols.append(col)
        if col:
            low = max(col)
            low_owner[low] = j
            paired.update((low, j))
            if val[order[low]] != val[c]:
                counts[C.dim(order[low])] += 1
                counts[C.dim(c)] += 1
    for j, c in enumerate(order):
        if j not in paired:
            counts[C.dim(c)] += 1
    return counts


def vpath_counts(C, pair, crit1, crit2):
    """{(1-saddle cell, 2-saddle cell): number of V-paths}, by enumeration downward from 2-saddles.

    A path leaves a quad through any facet other than the one the quad is paired with; at a
    1-cell it ends if the cell is critical, continues into the quad the cell is paired with,
    and is abandoned if the cell is paired with a vertex.
    """
    pd = pairs_dict(pair)
    crit1 = set(int(c) for c in crit1)
    counts = defaultdict(int)
    for t in crit2:
        t = int(t)
        stack = [(t, None)]
        while stack:
            q, excluded = stack.pop()
            for e in C.facets(q):
                if e == excluded:
                    continue
                if e in crit1:
                    counts[(e, t)] += 1
                    continue
                p = pd[e]
                if C.dim(p) == 2:
                    stack.append((p, e))
    return dict(counts)


def sparse_mul(X, Y):
    out = defaultdict(int)
    rows_y = defaultdict(list)
    for (r, c), v in Y.items():
        rows_y[r].append((c, v))
    for (r, k), v in X.items():
        for c, w in rows_y.get(k, ()):
            out[(r, c)] += v * w
    return {k: v for k, v in out.items() if v}


def paper_iterated_product(mn):
    """Sec. 3.3: A* = sum_k A B^k (iterate while the product is non-zero), D* = A* B* + D."""
    to_d = lambda t: {(int(r), int(c)): int(m) for r, c, m in zip(*t)}
    A, B, Bs, D = (to_d(mn[k]) for k in oracle.MINOR_NAMES)
    Astar = defaultdict(int)
    Ak = dict(A)
    iters = 0
    while Ak:
        iters += 1
        for k, v in Ak.items():
            Astar[k] += v
        Ak = sparse_mul(Ak, B)
    Dstar = defaultdict(int, sparse_mul(dict(Astar), Bs))
    for k, v in D.items():
        Dstar[k] += v
    return {k: v for k, v in Dstar.items() if v}, iters


# ----------------------------------------------------------------------------------
# tests
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("f", _fields_small(), ids=lambda f: "x".join(map(str, f.shape)))
def test_invariants_and_persistence(f):
    C = Complex(_dims(f))
    pair = oracle.gradient(f)
    rank = vertex_rank(f)
    pd = pairs_dict(pair)
    maxv = lambda c: max(C.vertices(c), key=lambda v: rank[v])
    for a, b in pd.items():
        assert pd[b] == a, "pairing not symmetric"
        lo, hi = (a, b) if C.dim(a) < C.dim(b) else (b, a)
        assert C.dim(hi) == C.dim(lo) + 1
        assert lo in C.facets(hi), "pair is not facet/cofacet"
        assert maxv(lo) == maxv(hi), "pair leaves a lower star"
    # acyclicity of the modified Hasse diagram: pair edges up, other facet edges down
    succ = defaultdict(list)
    indeg = defaultdict(int)
    for c in C.cells():
        for x in C.facets(c):
            if pd.get(x) == c:
                succ[x].append(c)
                indeg[c] += 1
            else:
                succ[c].append(x)
                indeg[x] += 1
    queue = [c for c in C.cells() if indeg[c] == 0]
    seen = 0
    while queue:
        c = queue.pop()
        seen += 1
        for d in succ[c]:
            indeg[d] -= 1
            if indeg[d] == 0:
                queue.append(d)
    assert seen == C.ncells(), "closed V-path found"
    counts, _ = oracle.critical(_dims(f), pair)
    assert counts[0] - counts[1] + counts[2] - counts[3] == 1
    assert list(counts) == persistence_critical_counts(f)


@pytest.mark.parametrize("seed", range(6))
def test_vertex_pairs_are_steepest_descent(seed):
    f = random_field((5, 6, 7), seed, "ties" if seed % 2 else "normal")
    nz, ny, nx = f.shape
    C = Complex(_dims(f))
    rank = vertex_rank(f)
    pair = oracle.gradient(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                v = C.vid(x, y, z)
                lower = []
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    X, Y, Z = x + dx, y + dy, z + dz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz and rank[C.vid(X, Y, Z)] < rank[v]:
                        lower.append((rank[C.vid(X, Y, Z)], (X, Y, Z)))
                vc = C.cid((2 * x, 2 * y, 2 * z))
                if not lower:
                    assert pair[vc] == NONE
                else:
                    X, Y, Z = min(lower)[1]
                    assert pair[vc] == C.cid((x + X, y + Y, z + Z))  # the edge between them


def test_euler_on_medium_fields():
    for f in (fields.grf((20, 24, 28), 3.0, seed=5), fields.batch_volume(7, lo=16, hi=24),
              fields.gaussian_blobs(n=24, n_blobs=6, sigma_range=(2, 5), seed=3)):
        counts, _ = oracle.critical(_dims(f), oracle.gradient(f))
        assert counts[0] - counts[1] + counts[2] - counts[3] == 1


def _grid(n):
    i = np.arange(n, dtype=np.float64)
    return np.meshgrid(i, i, i, indexing="ij")  # z, y, x


@pytest.mark.parametrize("n", [5, 8, 9])
def test_analytic_fields(n):
    z, y, x = _grid(n)
    c = (n - 1) / 2.0
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    for f, want in ((r2, [1, 0, 0, 0]),
                    (0.3 * x + 0.5 * y + 0.7 * z, [1, 0, 0, 0]),
                    (-r2, [8, 12, 6, 1])):
        f = np.ascontiguousarray(f.astype(np.float32))
        counts, _ = oracle.critical(_dims(f), oracle.gradient(f))
        assert list(counts) == want


def test_cosine_lattice_counts():
    """32^3 lattice: per axis minima at 8 and 24 and an interior maximum at 16 -> (8, 12, 6, 1)."""
    f = fields.cosine_lattice()
    counts, _ = oracle.critical(_dims(f), oracle.gradient(f))
    assert list(counts) == [8, 12, 6, 1]


@pytest.mark.parametrize("seed", range(8))
def test_dstar_matches_vpath_enumeration_and_paper_products(seed):
    shp = [(4, 4, 4), (5, 5, 4), (3, 6, 5), (6, 5, 5)][seed % 4]
    f = random_field(shp, 100 + seed, "normal" if seed < 6 else "ties")
    d = _dims(f)
    C = Complex(d)
    r = oracle.compute_all(f)
    s1, s2 = r["lists"][1], r["lists"][2]
    rows, cols, cnt = r["dstar"]
    got = {(int(s1[a]), int(s2[b])): int(c) for a, b, c in zip(rows, cols, cnt)}
    assert got == vpath_counts(C, r["pair"], s1, s2)
    prod, iters = paper_iterated_product(r["minor"])
    assert {(int(s1[a]), int(s2[b])): v for (a, b), v in prod.items()} == got
    assert iters == r["n_iter"]


def test_adjacent_saddles_two_node_component():
    """Fig. "msc-max-min-dag" (c): a 2-saddle adjacent to a 1-saddle gives a direct DAG edge."""
    found = 0
    for seed in range(40):
        f = random_field((4, 4, 4), 500 + seed)
        r = oracle.compute_all(f)
        C = Complex(_dims(f))
        s1 = [int(c) for c in r["lists"][1]]
        s2 = [int(c) for c in r["lists"][2]]
        rows, cols, cnt = r["dstar"]
        got = {(s1[a], s2[b]): int(c) for a, b, c in zip(rows, cols, cnt)}
        D = {(s1[a], s2[b]): int(m) for a, b, m in zip(*r["minor"]["D"])}
        for t in s2:
            for e in C.facets(t):
                if e in set(s1):
                    found += 1
                    assert D.get((e, t), 0) >= 1 and got[(e, t)] >= 1
    assert found > 0


@pytest.mark.parametrize("seed", range(4))
def test_min_labels_are_steepest_descent(seed):
    f = random_field((6, 5, 7), 200 + seed, "ties" if seed % 2 else "normal")
    nz, ny, nx = f.shape
    C = Complex(_dims(f))
    rank = vertex_rank(f)
    r = oracle.compute_all(f, with_minor=False, with_dstar=False)
    vmin = r["vertex_min"].reshape(-1)
    for v0 in range(nx * ny * nz):
        v = v0
        while True:
            x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
            best = None
            for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                X, Y, Z = x + dx, y + dy, z + dz
                if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                    w = C.vid(X, Y, Z)
                    if rank[w] < rank[v] and (best is None or rank[w] < rank[best]):
                        best = w
            if best is None:
                break
            v = best
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        assert vmin[v0] == C.cid((2 * x, 2 * y, 2 * z))
    # 1-saddle arcs are the destinations of the edge's two vertices, lower coordinate first
    for i, e in enumerate(r["lists"][1]):
        a, b = sorted(C.vertices(int(e)))
        assert (r["min_arcs"][2 * i], r["min_arcs"][2 * i + 1]) == (vmin[a], vmin[b])


@pytest.mark.parametrize("seed", range(4))
def test_max_labels_properties(seed):
    f = random_field((6, 7, 5), 300 + seed)
    nz, ny, nx = f.shape
    C = Complex(_dims(f))
    rank = vertex_rank(f)
    r = oracle.compute_all(f, with_minor=False, with_dstar=False)
    pd = pairs_dict(r["pair"])
    cmax = r["cube_max"]
    maxes = set(int(c) for c in r["lists"][3])
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                lab = int(cmax[z, y, x])
                if x == nx - 1 or y == ny - 1 or z == nz - 1:
                    assert lab == NONE
                    continue
                c = C.cid((2 * x + 1, 2 * y + 1, 2 * z + 1))
                if c in maxes:
                    assert lab == c
                    continue
                assert lab == NONE or lab in maxes
                if lab != NONE:
                    top = lambda cell: max(rank[v] for v in C.vertices(cell))
                    assert top(lab) >= top(c)
                q = pd[c]
                other = [k for k in C.cofacets(q) if k != c]
                if not other:
                    assert lab == NONE
                else:
                    ox, oy, oz = (v // 2 for v in C.coords(other[0]))
                    assert lab == int(cmax[oz, oy, ox])
    for i, q in enumerate(r["lists"][2]):
        cc = C.coords(int(q))
        k = [a for a in range(3) if cc[a] % 2 == 0][0]
        for side, s in enumerate((-1, 1)):
            d = list(cc)
            d[k] += s
            want = int(cmax[d[2] // 2, d[1] // 2, d[0] // 2]) if C.inside(d) else NONE
            assert r["max_arcs"][2 * i + side] == want


@pytest.mark.parametrize("seed", range(4))
def test_reachable_and_junctions(seed):
    f = random_field((5, 6, 5), 400 + seed)
    nz, ny, nx = f.shape
    C = Complex(_dims(f))
    r = oracle.compute_all(f)
    pd = pairs_dict(r["pair"])
    s1 = set(int(c) for c in r["lists"][1])
    s2 = set(int(c) for c in r["lists"][2])

    def out(e):
        res = []
        for q in C.cofacets(e):
            if pd.get(e) == q:
                continue
            if q in s2:
                res.append(q)
            elif C.dim(pd[q]) == 1:
                res.append(pd[q])
        return res

    vis = r["visited"]

    def visited(e):
        cx, cy, cz = C.coords(e)
        axis = 0 if cx & 1 else (1 if cy & 1 else 2)
        return bool((vis[cz // 2, cy // 2, cx // 2] >> axis) & 1)

    # every 1-cell on a V-path between saddles is reachable; the set is closed under out-edges
    nodes = [e for e in C.cells() if C.dim(e) == 1 and (e in s1 or C.dim(pd[e]) == 2)]
    for e in nodes:
        if visited(e):
            for w in out(e):
                assert w in s2 or visited(w)
    for e in s1:
        assert visited(e)
    marked = sum(int(np.unpackbits(np.array([b], dtype=np.uint8)).sum()) for b in vis.reshape(-1))
    assert marked == sum(visited(e) for e in nodes)
    want_j = sorted(e for e in nodes if visited(e) and e not in s1 and len(out(e)) > 1)
    assert [int(j) for j in r["junctions"]] == want_j


def test_nan_rejected_and_infinities_ordered():
    f = random_field((3, 3, 3), 1)
    g = f.copy()
    g[1, 1, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.gradient(g)
    assert e.value.status == 2
    h = f.copy()
    h[0, 0, 0] = -np.inf
    h[2, 2, 2] = np.inf
    counts, _ = oracle.critical(_dims(h), oracle.gradient(h))
    assert counts[0] - counts[1] + counts[2] - counts[3] == 1
    # -0 and +0 compare equal: ties are broken by vertex index only
    z = np.zeros((2, 2, 2), dtype=np.float32)
    z[0, 0, 0] = -0.0
    assert list(oracle.critical((2, 2, 2), oracle.gradient(z))[0]) == [1, 0, 0, 0]


def _decode_packed_words(dims, words):
    """The partner of every cell, read from packed words by the word layout's definition (one
    uint32 per vertex; vertex (x,y,z) owns the cells (2x+a, 2y+b, 2z+c), slot s = a + 2b + 4c,
    3-bit code in bits [3s, 3s+3): 0 critical, 1..6 partner one step along -x, +x, -y, +y, -z, +z
    of the refined grid, 7 no such cell).  Returns (cell ids, partner ids or NONE) for every
    existing cell, and whether every non-existing cell carries code 7."""
    nx, ny, nz = (int(v) for v in dims)
    rx, ry, rz = 2 * nx - 1, 2 * ny - 1, 2 * nz - 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    words = words.astype(np.int64)
    step = {1: (-1, 0, 0), 2: (1, 0, 0), 3: (0, -1, 0), 4: (0, 1, 0), 5: (0, 0, -1), 6: (0, 0, 1)}
    cells, partners, off_grid_ok = [], [], True
    for s in range(8):
        a, b, c = s & 1, (s >> 1) & 1, (s >> 2) & 1
        cx, cy, cz = 2 * x + a, 2 * y + b, 2 * z + c
        code = (words >> (3 * s)) & 7
        inside = (cx < rx) & (cy < ry) & (cz < rz)
        off_grid_ok &= bool(np.all(code[~inside] == 7))
        cid = cx + rx * (cy + ry * cz)
        part = np.full(code.shape, 0xFFFFFFFF, dtype=np.int64)
        for k, (dx, dy, dz) in step.items():
            sel = code == k
            part[sel] = ((cx + dx) + rx * ((cy + dy) + ry * (cz + dz)))[sel]
        bad = inside & (code == 7)  # an existing cell must be critical or paired
        part[bad] = -1
        cells.append(cid[inside])
        partners.append(part[inside])
    return np.concatenate(cells), np.concatenate(partners), off_grid_ok


@pytest.mark.parametrize("seed", range(4))
def test_packed_words_decode_to_the_gradient_pairs(seed):
    """The packed-word convention (the library's exchange format) against the pairs it encodes:
    every word of oracle.pack, decoded by the layout's definition, names each cell's partner as
    oracle.gradient does; every cell of the refined grid appears exactly once."""
    shapes = [(5, 6, 7), (3, 9, 4), (8, 8, 2), (2, 5, 11)]
    for kind in ("normal", "ties"):
        f = random_field(shapes[seed], 300 + seed, kind)
        dims = (f.shape[2], f.shape[1], f.shape[0])
        pair = oracle.gradient(f)
        cells, partners, off_grid_ok = _decode_packed_words(dims, oracle.pack(dims, pair))
        assert off_grid_ok
        assert np.array_equal(np.sort(cells), np.arange(pair.size))
        assert np.array_equal(partners, pair[cells].astype(np.int64))


def _cell_coords(dims, c):
    nx, ny, nz = dims
    rx, ry = 2 * nx - 1, 2 * ny - 1
    return (int(c) % rx, (int(c) // rx) % ry, int(c) // (rx * ry))


def _facets(dims, c):
    """Facets of a cell by the definition: move one odd coordinate by -1 or +1."""
    nx, ny, nz = dims
    rx, ry = 2 * nx - 1, 2 * ny - 1
    cc = _cell_coords(dims, c)
    out = set()
    for a in range(3):
        if cc[a] % 2:
            for s in (-1, 1):
                d = list(cc)
                d[a] += s
                out.add(d[0] + rx * (d[1] + ry * d[2]))
    return out


def _dim(dims, c):
    return sum(v % 2 for v in _cell_coords(dims, c))


@pytest.mark.parametrize("seed", range(4))
def test_arc_cells_are_the_v_paths_of_the_arcs(seed):
    """Every arc's cells form the V-path of Sec. 2.2 between its saddle and its extremum: a
    descending path alternates a vertex and the edge it is paired with, each next vertex being the
    other facet of that edge; an ascending path alternates a cube and the quad it is paired with
    (a facet of the cube), each next cube being the other cofacet of that quad.  Paths end at an
    unpaired extremum equal to the arc lists' endpoint, or, ascending, at a quad with no cube beyond
    it (endpoint NONE); no cell repeats."""
    shapes = [(5, 6, 7), (3, 9, 4), (8, 8, 2), (2, 5, 11)]
    for kind in ("normal", "ties"):
        f = random_field(shapes[seed], 400 + seed, kind)
        dims = (f.shape[2], f.shape[1], f.shape[0])
        nx, ny, nz = dims
        rx, ry, rz = 2 * nx - 1, 2 * ny - 1, 2 * nz - 1
        pair = oracle.gradient(f)
        _, lists = oracle.critical(dims, pair)
        _, _, amin, amax = oracle.extremum(dims, pair, lists[1], lists[2])
        off, cells = oracle.arc_cells(dims, pair, lists[1], lists[2])
        n1, n2 = len(lists[1]), len(lists[2])
        assert len(off) == 2 * (n1 + n2) + 1 and off[-1] == len(cells)
        NONE = 0xFFFFFFFF
        for a in range(2 * (n1 + n2)):
            path = [int(c) for c in cells[off[a]:off[a + 1]]]
            assert len(set(path)) == len(path)
            if a < 2 * n1:
                e = int(lists[1][a // 2])
                assert path[0] == e and len(path) % 2 == 0
                lo, hi = sorted(_facets(dims, e))
                assert path[1] == (hi if a % 2 else lo)  # lower-coordinate vertex first
                for k in range(1, len(path) - 1, 2):
                    v, ed, w = path[k], path[k + 1], path[k + 2]
                    assert _dim(dims, v) == 0 and int(pair[v]) == ed
                    assert w in _facets(dims, ed) and w != v
                assert int(pair[path[-1]]) == NONE and path[-1] == int(amin[a])
            else:
                b = a - 2 * n1
                q = int(lists[2][b // 2])
                assert path[0] == q
                if len(path) == 1:  # no cube on that side
                    assert int(amax[b]) == NONE
                    continue
                assert q in _facets(dims, path[1])
                qc = _cell_coords(dims, q)
                axis = [qc[i] % 2 for i in range(3)].index(0)
                assert _cell_coords(dims, path[1])[axis] - qc[axis] == (1 if b % 2 else -1)
                for k in range(1, len(path) - 1, 2):
                    c, quad = path[k], path[k + 1]
                    assert _dim(dims, c) == 3 and int(pair[c]) == quad and quad in _facets(dims, c)
                    if k + 2 < len(path):
                        nxt = path[k + 2]
                        assert quad in _facets(dims, nxt) and nxt != c
                last = path[-1]
                if _dim(dims, last) == 3:
                    assert int(pair[last]) == NONE and last == int(amax[b])
                else:  # left the domain through this quad: it has one cofacet cube
                    lc = _cell_coords(dims, last)
                    ext = (rx, ry, rz)
                    even = [i for i in range(3) if lc[i] % 2 == 0][0]
                    inside = [0 <= lc[even] + s < ext[even] for s in (-1, 1)]
                    assert sum(inside) == 1 and int(amax[b]) == NONE


def vpath_cell_lists(C, pair, crit1, crit2):
    """{(1-saddle cell, 2-saddle cell): [cell sequence of each V-path]}, enumerated downward from
    every 2-saddle as in vpath_counts, each sequence read from the 1-saddle up: s, then the quad
    and the 1-cell of each step (the quad the 1-cell is paired with), then t."""
    pd = pairs_dict(pair)
    crit1 = set(int(c) for c in crit1)
    out = defaultdict(list)
    for t in crit2:
        t = int(t)
        stack = [(t, None, [t])]
        while stack:
            q, excluded, down = stack.pop()
            for e in C.facets(q):
                if e == excluded:
                    continue
                if e in crit1:
                    out[(e, t)].append([e] + down[::-1])
                    continue
                p = pd[e]
                if C.dim(p) == 2:
                    stack.append((p, e, down + [e, p]))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_ss_arc_cells_are_the_single_v_paths(seed):
    """Every D* entry of count 1 gets the cells of its one V-path (enumerated downward from the
    2-saddle, independently of the oracle's upward walk), every other entry none; the enumeration
    also reproduces every count."""
    if seed < 4:
        f = random_field([(6, 6, 6), (5, 7, 8), (8, 6, 5), (4, 9, 7)][seed], 700 + seed,
                         "normal" if seed % 2 == 0 else "ties")
    else:
        f = fields.gaussian_blobs(n=14, n_blobs=5, sigma_range=(2, 4), seed=60 + seed)
    d = _dims(f)
    C = Complex(d)
    r = oracle.compute_all(f)
    s1, s2 = r["lists"][1], r["lists"][2]
    rows, cols, cnt = r["dstar"]
    off, cells = oracle.ss_arc_cells(d, r["pair"], s1, s2, r["dstar"])
    assert len(off) == len(cnt) + 1 and off[-1] == len(cells)
    paths = vpath_cell_lists(C, r["pair"], s1, s2)
    assert sum(len(v) for v in paths.values()) == int(np.sum(cnt))
    n_one = n_long = 0
    for k, (a, b, c) in enumerate(zip(rows, cols, cnt)):
        key = (int(s1[a]), int(s2[b]))
        got = [int(x) for x in cells[off[k]:off[k + 1]]]
        assert len(paths[key]) == int(c)
        if int(c) == 1:
            assert got == paths[key][0]
            n_one += 1
            n_long += len(got) > 2
        else:
            assert got == []
    assert n_one > 0 and n_long > 0


def test_packed_at_matches_full_pack():
    f = fields.grf((9, 10, 11), 3.0, seed=9)
    pair = oracle.gradient(f)
    full = oracle.pack(_dims(f), pair).reshape(-1)
    verts = np.arange(full.size)
    assert np.array_equal(oracle.packed_at(f, verts), full)


@pytest.mark.parametrize("seed", range(3))
def test_lazy_sampled_queries_equal_whole_volume(seed):
    """The sampled (lazily paired) oracle queries used on full-size volumes reproduce the
    whole-volume oracle: pairs, labels, DAG-node facts and D* rows."""
    f = [fields.grf((30, 31, 32), 3.0, seed=40 + seed), random_field((9, 10, 11), 41 + seed, "ties"),
         fields.gaussian_blobs(n=28, n_blobs=6, sigma_range=(2, 6), seed=42 + seed)][seed]
    r = oracle.compute_all(f)
    s1, s2 = r["lists"][1], r["lists"][2]
    cells = np.arange(0, len(r["pair"]), 5, dtype=np.uint32)
    assert np.array_equal(oracle.lazy_pairs(f, cells), r["pair"][cells])
    v = np.arange(0, f.size, 3)
    assert np.array_equal(oracle.lazy_vertex_min(f, v), r["vertex_min"].reshape(-1)[v])
    assert np.array_equal(oracle.lazy_cube_max(f, v), r["cube_max"].reshape(-1)[v])
    rows = oracle.lazy_dstar_rows(f, s1)
    R, C, K = r["dstar"]
    full = {}
    for a, b, k in zip(R, C, K):
        full.setdefault(int(s1[a]), {})[int(s2[b])] = int(k)
    assert all(rows[int(c)] == full.get(int(c), {}) for c in s1)
    C3 = Complex(_dims(f))
    ones = np.array([c for c in range(C3.ncells()) if C3.dim(c) == 1], dtype=np.uint32)
    facts = oracle.lazy_nodes(f, ones)
    jset = set(int(j) for j in r["junctions"])
    vis = r["visited"]
    for c, (node, crit, deg) in zip(ones, facts):
        cx, cy, cz = C3.coords(int(c))
        axis = 0 if cx & 1 else (1 if cy & 1 else 2)
        visited = bool((vis[cz // 2, cy // 2, cx // 2] >> axis) & 1)
        assert (int(c) in jset) == (visited and node and not crit and deg > 1)
        assert crit == (r["pair"][c] == 0xFFFFFFFF)


# ----------------------------------------------------------------------------------
# persistence-ordered simplification (Sec. 4)
# ----------------------------------------------------------------------------------
def _replay_simplification(sk, threshold):
    """Brute force, written from the cancellation rule: repeatedly take the least valid arc (consecutive
    index, both ends alive, exactly one arc between them) by (persistence, upper cell, lower cell),
    while its persistence <= threshold; reroute every descending neighbour a of the upper node p
    (a != q) to every ascending neighbour b of the lower node q (b != p) with m(p,a) * m(q,b) new
    arcs, then delete p and q.  Checks the Euler characteristic after every cancellation."""
    index, value, cell = [int(i) for i in sk["index"]], [float(v) for v in sk["value"]], [int(c) for c in sk["cell"]]
    n = len(index)
    adj = [dict() for _ in range(n)]
    for u, v, m in zip(sk["arc_u"], sk["arc_v"], sk["arc_mult"]):
        u, v, m = int(u), int(v), int(m)
        adj[u][v] = adj[u].get(v, 0) + m
        adj[v][u] = adj[v].get(u, 0) + m
    alive = [True] * n
    euler = lambda: sum((-1) ** index[i] for i in range(n) if alive[i])
    e0 = euler()
    log = []
    while True:
        best = None
        for p in range(n):
            if not alive[p]:
                continue
            for q, m in adj[p].items():
                if alive[q] and index[p] == index[q] + 1 and m == 1:
                    key = (abs(value[p] - value[q]), cell[p], cell[q])
                    if key[0] <= threshold and (best is None or key < best[0]):
                        best = (key, p, q)
        if best is None:
            break
        key, p, q = best
        down = [(a, m) for a, m in adj[p].items() if a != q and index[a] == index[q]]
        up = [(b, m) for b, m in adj[q].items() if b != p and index[b] == index[p]]
        for a, ma in down:
            for b, mb in up:
                adj[b][a] = adj[b].get(a, 0) + ma * mb
                adj[a][b] = adj[b][a]
        for x in (p, q):
            for y in list(adj[x]):
                del adj[y][x]
            adj[x].clear()
            alive[x] = False
        log.append((p, q, key[0]))
        assert euler() == e0
    arcs = sorted((u, v, m) for u in range(n) for v, m in adj[u].items() if u < v)
    return log, alive, arcs


@pytest.mark.parametrize("seed", range(4))
def test_simplification_matches_brute_force_replay(seed):
    shapes = [(4, 5, 6), (3, 7, 4), (6, 6, 2), (2, 5, 9)]
    for kind in ("normal", "ties"):
        f = random_field(shapes[seed], 500 + seed, kind)
        sk = oracle.skeleton(f)
        pers = np.abs(sk["value"][sk["arc_u"]] - sk["value"][sk["arc_v"]])
        for threshold in (0.0, float(np.median(pers)) if len(pers) else 0.0, 1e9):
            r = oracle.simplify(sk, threshold)
            log, alive, arcs = _replay_simplification(sk, threshold)
            assert [(int(a), int(b)) for a, b in zip(r["upper"], r["lower"])] == [(p, q) for p, q, _ in log]
            assert np.allclose(r["persistence"], [x for _, _, x in log])
            assert list(r["alive"]) == alive
            assert sorted(zip(r["arc_u"].tolist(), r["arc_v"].tolist(), r["arc_mult"].tolist())) == arcs


def test_simplification_two_wells_closed_form():
    """Two parabolic wells along x, depths 0 and 10, meeting at x = 15 where the barrier is 49: the
    complex is two minima and one 1-saddle, and the only pair, (saddle, the shallower minimum), has
    persistence 49 - 10 = 39: it is cancelled exactly when the threshold reaches 39."""
    x = np.arange(31)[None, None, :]
    y = np.arange(9)[None, :, None]
    z = np.arange(9)[:, None, None]
    f = (np.minimum((x - 8.0) ** 2, (x - 22.0) ** 2 + 10.0) + (y - 4.0) ** 2 + (z - 4.0) ** 2).astype(np.float32)
    sk = oracle.skeleton(f)
    assert list(np.bincount(sk["index"], minlength=4)) == [2, 1, 0, 0]
    r = oracle.simplify(sk, 38.999)
    assert len(r["upper"]) == 0
    r = oracle.simplify(sk, 39.0)
    assert len(r["upper"]) == 1 and r["persistence"][0] == 39.0
    assert sk["value"][r["lower"][0]] == 10.0 and sk["index"][r["upper"][0]] == 1
    assert list(np.bincount(sk["index"][r["alive"]], minlength=4)) == [1, 0, 0, 0] and len(r["arc_u"]) == 0


def test_simplification_cosine_lattice_closed_form():
    """The cosine lattice's pairs differ by one cosine step, persistence 2 (up to its 1e-3 noise): below
    it the complex stays (8, 12, 6, 1) with all its arcs; above it every pair cancels and a single
    minimum is left, the complex of the box."""
    f = fields.cosine_lattice()
    sk = oracle.skeleton(f)
    assert list(np.bincount(sk["index"], minlength=4)) == [8, 12, 6, 1]
    r = oracle.simplify(sk, 1.99)
    assert len(r["upper"]) == 0 and len(r["arc_u"]) == len(sk["arc_u"])
    r = oracle.simplify(sk, 2.01)
    assert len(r["upper"]) == 13 and np.all(np.abs(r["persistence"] - 2.0) < 2e-3)
    assert list(np.bincount(sk["index"][r["alive"]], minlength=4)) == [1, 0, 0, 0] and len(r["arc_u"]) == 0


def _replay_rounds(sk, threshold):
    """Brute force of the round rule: each round, the valid arcs whose key is the least among the valid
    arcs with an endpoint within two links (breadth-first distances) of one of theirs are cancelled
    together; their footprints (ends and neighbours) must be disjoint."""
    index, value, cell = [int(i) for i in sk["index"]], [float(v) for v in sk["value"]], [int(c) for c in sk["cell"]]
    n = len(index)
    adj = [dict() for _ in range(n)]
    for u, v, m in zip(sk["arc_u"], sk["arc_v"], sk["arc_mult"]):
        u, v, m = int(u), int(v), int(m)
        adj[u][v] = adj[u].get(v, 0) + m
        adj[v][u] = adj[v].get(u, 0) + m
    alive = [True] * n
    rounds = []
    while True:
        valid = {}
        for p in range(n):
            for q, m in adj[p].items():
                if alive[p] and alive[q] and index[p] == index[q] + 1 and m == 1:
                    k = (abs(value[p] - value[q]), cell[p], cell[q])
                    if k[0] <= threshold:
                        valid[(p, q)] = k

        def near(x):  # nodes within two links of x
            seen, front = {x}, [x]
            for _ in range(2):
                front = [y for z in front for y in adj[z] if y not in seen]
                seen.update(front)
            return seen

        chosen = []
        for (p, q), k in valid.items():
            zone = near(p) | near(q)
            if all(k2 >= k for (a, b), k2 in valid.items() if a in zone or b in zone):
                chosen.append((p, q))
        if not chosen:
            break
        fps = [{p, q} | set(adj[p]) | set(adj[q]) for p, q in chosen]
        assert sum(len(x) for x in fps) == len(set().union(*fps))
        for p, q in chosen:
            down = [(a, m) for a, m in adj[p].items() if a != q and index[a] == index[q]]
            up = [(b, m) for b, m in adj[q].items() if b != p and index[b] == index[p]]
            for a, ma in down:
                for b, mb in up:
                    adj[b][a] = adj[b].get(a, 0) + ma * mb
                    adj[a][b] = adj[b][a]
            for x in (p, q):
                for y in list(adj[x]):
                    del adj[y][x]
                adj[x].clear()
                alive[x] = False
        rounds.append(sorted(chosen))
    arcs = sorted((u, v, m) for u in range(n) for v, m in adj[u].items() if u < v)
    return rounds, alive, arcs


@pytest.mark.parametrize("seed", range(3))
def test_simplification_rounds_match_brute_force_and_the_serial_order(seed):
    """The round rule against its brute-force replay (round by round); on these fields it also ends
    in exactly the complex that the serial order gives (same survivors, arcs and cancelled pairs)."""
    shapes = [(4, 5, 6), (3, 7, 4), (6, 6, 3)]
    for kind in ("normal", "ties"):
        f = random_field(shapes[seed], 600 + seed, kind)
        sk = oracle.skeleton(f)
        pers = np.abs(sk["value"][sk["arc_u"]] - sk["value"][sk["arc_v"]])
        for threshold in (0.0, float(np.median(pers)) if len(pers) else 0.0, 1e9):
            r = oracle.simplify(sk, threshold, rounds=True)
            rounds, alive, arcs = _replay_rounds(sk, threshold)
            assert r["n_rounds"] == len(rounds)
            got = [sorted((int(a), int(b)) for a, b, k in zip(r["upper"], r["lower"], r["round"]) if k == i)
                   for i in range(r["n_rounds"])]
            assert got == rounds
            assert list(r["alive"]) == alive
            assert sorted(zip(r["arc_u"].tolist(), r["arc_v"].tolist(), r["arc_mult"].tolist())) == arcs
            s = oracle.simplify(sk, threshold)
            assert np.array_equal(s["alive"], r["alive"])
            assert set(zip(s["upper"].tolist(), s["lower"].tolist())) == set(zip(r["upper"].tolist(), r["lower"].tolist()))


def test_simplification_rounds_closed_forms():
    x = np.arange(31)[None, None, :]
    y = np.arange(9)[None, :, None]
    z = np.arange(9)[:, None, None]
    f = (np.minimum((x - 8.0) ** 2, (x - 22.0) ** 2 + 10.0) + (y - 4.0) ** 2 + (z - 4.0) ** 2).astype(np.float32)
    sk = oracle.skeleton(f)
    assert len(oracle.simplify(sk, 38.999, rounds=True)["upper"]) == 0
    r = oracle.simplify(sk, 39.0, rounds=True)
    assert r["n_rounds"] == 1 and r["persistence"].tolist() == [39.0]
    sk = oracle.skeleton(fields.cosine_lattice())
    assert oracle.simplify(sk, 1.99, rounds=True)["n_rounds"] == 0
    r = oracle.simplify(sk, 2.01, rounds=True)
    assert len(r["upper"]) == 13 and list(np.bincount(sk["index"][r["alive"]], minlength=4)) == [1, 0, 0, 0]
