"""Full-size parity on the bench workload (256^3 k^-3 GRF) and the 512^3 Gaussian-blob field,
in the configuration bench.py times: one plan with default options, on the current stream, and
its third msc_compute -- the replayed CUDA graph with the autotuned lower-star tile, the
saddle-extremum branch beside the critical path, and the path-count method the plan chose after
its first pass (row-wise products on the shallow GRF minor, junction waves on the deep blob
minor).  The oracle cannot run these volumes whole in test time, so it checks sampled outputs
one by one (its lower-star pairs are computed lazily, one vertex's star at a time), and
properties that hold at any size cover the rest."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.gpu_util import csr_to_coo, dims_of, gpu_field, msc, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NONE = 0xFFFFFFFF


def _run(f):
    m = msc()
    plan = m.Plan(dims_of(f))
    d = gpu_field(f)
    for _ in range(3):  # synchronised first pass, graph capture, then a replay (as the bench)
        m.msc_compute(plan, d)
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    vis, levels = m.msc_reachability(plan)
    junc = m.msc_junctions(plan)
    rp, col, cnt = m.msc_saddle_arcs(plan)
    return dict(words=to_np(m.msc_gradient_words(plan)), counts=counts, cells=[to_np(c) for c in cells],
                amin=to_np(amin), amax=to_np(amax), vmin=to_np(vmin).reshape(-1), cmax=to_np(cmax).reshape(-1),
                visited=to_np(vis), junctions=to_np(junc), rowptr=to_np(rp), col=to_np(col), cnt=to_np(cnt),
                stats=m.msc_get_stats(plan))


def _check(f, r, n_samples, seed, n_rows=None):
    rng = np.random.default_rng(seed)
    nz, ny, nx = f.shape
    rx, ry = 2 * nx - 1, 2 * ny - 1
    counts = r["counts"]
    # (a1) packed words at sampled vertices, including a box that straddles CTA tiles
    z, y, x = np.meshgrid(np.arange(20, 30), np.arange(5, 15), np.arange(25, 70), indexing="ij")
    verts = np.concatenate([rng.integers(0, f.size, size=n_samples), (x + nx * (y + ny * z)).reshape(-1),
                            [0, f.size - 1]])
    assert np.array_equal(r["words"].reshape(-1)[verts], oracle.packed_at(f, verts))
    # (a2) lists: increasing, of the right dimension, critical in the words, complete in count
    assert counts[0] - counts[1] + counts[2] - counts[3] == 1
    flat = r["words"].reshape(-1)
    total = 0
    for k in range(4):
        c = r["cells"][k].astype(np.int64)
        assert len(c) == counts[k] and np.all(np.diff(c) > 0)
        cx, cy, cz = c % rx, (c // rx) % ry, c // (rx * ry)
        assert np.all((cx & 1) + (cy & 1) + (cz & 1) == k)
        slot = (cx & 1) + 2 * (cy & 1) + 4 * (cz & 1)
        assert np.all(((flat[(cx // 2) + nx * ((cy // 2) + ny * (cz // 2))] >> (3 * slot)) & 7) == 0)
        total += len(c)
    assert int((((flat[:, None] >> (3 * np.arange(8))[None, :]) & 7) == 0).sum()) == total
    # (a3) labels of sampled vertices and cubes, arcs of sampled saddles
    v = rng.integers(0, f.size, size=n_samples)
    assert np.array_equal(r["vmin"][v], oracle.lazy_vertex_min(f, v))
    assert np.array_equal(r["cmax"][v], oracle.lazy_cube_max(f, v))
    i1 = rng.integers(0, counts[1], size=min(counts[1], n_samples // 4))
    e = r["cells"][1][i1].astype(np.int64)
    ex, ey, ez = e % rx, (e // rx) % ry, e // (rx * ry)
    lo = (ex // 2) + nx * ((ey // 2) + ny * (ez // 2))
    hi = ((ex + 1) // 2) + nx * (((ey + 1) // 2) + ny * ((ez + 1) // 2))
    assert np.array_equal(r["amin"][2 * i1], oracle.lazy_vertex_min(f, lo))
    assert np.array_equal(r["amin"][2 * i1 + 1], oracle.lazy_vertex_min(f, hi))
    i2 = rng.integers(0, counts[2], size=min(counts[2], n_samples // 4))
    q = r["cells"][2][i2].astype(np.int64)
    qc = np.stack([q % rx, (q // rx) % ry, q // (rx * ry)], axis=1)
    for side, sgn in ((0, -1), (1, 1)):
        d = qc.copy()
        axis = np.argmax((qc & 1) == 0, axis=1)
        d[np.arange(len(d)), axis] += sgn
        ext = np.array([rx, ry, 2 * nz - 1])
        inside = np.all((d >= 0) & (d < ext), axis=1)
        owner = (d[:, 0] // 2) + nx * ((d[:, 1] // 2) + ny * (d[:, 2] // 2))
        want = np.where(inside, oracle.lazy_cube_max(f, np.where(inside, owner, 0)), NONE)
        assert np.array_equal(r["amax"][2 * i2 + side], want.astype(np.uint32))
    # (a4)/(a5) sampled junctions are visited, non-critical DAG nodes of out-degree > 1; sampled
    # visited nodes are DAG nodes whose successors are visited
    W = (nx + 31) // 32
    vis = r["visited"]

    def visited(cells):
        cells = cells.astype(np.int64)
        cx, cy, cz = cells % rx, (cells // rx) % ry, cells // (rx * ry)
        b, c = (cy & 1), (cz & 1)
        wi = ((((cz // 2) * 2 + c) * ny + cy // 2) * 2 + b) * W + ((cx // 2) >> 5)
        return ((vis[wi] >> ((cx // 2) & 31).astype(np.uint32)) & 1).astype(bool)

    j = r["junctions"]
    assert len(j) == r["stats"]["n_junctions"] and np.all(np.diff(j.astype(np.int64)) > 0)
    js = j[rng.integers(0, len(j), size=min(len(j), n_samples // 4))]
    facts = oracle.lazy_nodes(f, js)
    assert np.all(facts[:, 0] == 1) and np.all(facts[:, 1] == 0) and np.all(facts[:, 2] > 1)
    assert np.all(visited(js))
    assert np.all(visited(r["cells"][1]))  # every 1-saddle is a BFS seed
    # (a6) D* rows of sampled 1-saddles against the oracle's per-source path counts.  The row-wise
    # products defer a row to the next tier when its tables overflow: a row of more than 16 entries
    # cannot finish in tier 0, of more than 32 not in tier 0b, of more than 256 not in tier 1.  So
    # beside random rows, every row longer than 16 entries (up to 400 of them, the longest first)
    # is checked too.
    rp = r["rowptr"]
    n_rows = n_rows or n_samples // 8
    lens = np.diff(rp.astype(np.int64))
    long_rows = np.argsort(-lens, kind="stable")[:400]
    long_rows = long_rows[lens[long_rows] > 16]
    rows = np.unique(np.concatenate([rng.integers(0, counts[1], size=min(counts[1], n_rows)), long_rows]))
    want = oracle.lazy_dstar_rows(f, r["cells"][1][rows])
    for s in rows:
        a, b = int(rp[s]), int(rp[s + 1])
        got = {int(r["cells"][2][c]): int(k) for c, k in zip(r["col"][a:b], r["cnt"][a:b])}
        assert got == want[int(r["cells"][1][s])]
    assert int(rp[-1]) == r["stats"]["nnz_Dstar"]


def test_grf256_bench_workload():
    f = fields.config_field("grf256")
    r = _run(f)
    assert r["stats"]["path_count_method"] == 1  # the replay timed by the bench: row-wise products
    _check(f, r, n_samples=4000, seed=1, n_rows=2000)


def test_blobs512():
    f = fields.config_field("blobs512")
    r = _run(f)
    assert r["stats"]["path_count_method"] == 2  # a minor of ~200 levels: junction waves
    _check(f, r, n_samples=2000, seed=2)
