"""Saddle-saddle arc geometry (Sec. 3.3 / Sec. 3.5 "Data structure"): msc_saddle_arc_geometry and
msc_copy_to_host against the oracle's single V-paths of the D* entries with count 1, element by
element, after passes that counted paths row by row and by junction waves."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF
STAT_KEYS = ("path_count_method", "n_frontier_entries", "n_iter", "max_path_count", "nnz_Dstar", "ms_rows_kernel")


def _cases():
    out = [("cos32", fields.cosine_lattice()), ("grf40", fields.grf((40, 36, 44), 3.0, seed=12)),
           ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5)),
           ("blobs30", fields.gaussian_blobs(n=30, n_blobs=4, sigma_range=(3, 8), seed=17))]
    z, y, x = np.meshgrid(np.arange(9), np.arange(10), np.arange(11), indexing="ij")
    out.append(("ramp", (x + 2.0 * y + 3.0 * z).astype(np.float32)))  # no saddles: D* is empty
    for i, shp in enumerate([(2, 2, 2), (3, 5, 7), (9, 8, 33), (17, 16, 65)]):
        out.append((f"normal{shp}", random_field(shp, 1900 + i, "normal")))
        out.append((f"ties{shp}", random_field(shp, 1950 + i, "ties")))
    return out


def _want(f):
    r = oracle.compute_all(f)
    return oracle.ss_arc_cells(dims_of(f), r["pair"], r["lists"][1], r["lists"][2], r["dstar"])


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("name,f", _cases(), ids=[n for n, _ in _cases()])
def test_ss_arc_geometry_matches_oracle(name, f, method):
    m = msc()
    plan = m.Plan(dims_of(f), path_count_method=method)
    m.msc_compute(plan, gpu_field(f))
    before = m.msc_get_stats(plan)
    rp, col, cnt = (to_np(x).copy() for x in m.msc_saddle_arcs(plan))
    off, cells = m.msc_saddle_arc_geometry(plan)
    want_off, want_cells = _want(f)
    assert np.array_equal(to_np(off), want_off)
    assert np.array_equal(to_np(cells), want_cells)
    assert np.array_equal(m.msc_copy_to_host(plan, "ss_arc_offsets"), want_off)
    assert np.array_equal(m.msc_copy_to_host(plan, "ss_arc_cells"), want_cells)
    # the pass's D* and statistics are what they were (row-wise passes rerun the junction waves)
    after = m.msc_get_stats(plan)
    assert all(after[k] == before[k] for k in STAT_KEYS), [(k, before[k], after[k]) for k in STAT_KEYS]
    for a, b in zip((rp, col, cnt), m.msc_saddle_arcs(plan)):
        assert np.array_equal(a, to_np(b))


def test_ss_geometry_of_replayed_passes_follows_the_field():
    """Built once per pass and dropped by the next: after replays of two fields on one plan (the
    method chosen automatically), each query returns the current field's arcs."""
    m = msc()
    a = fields.gaussian_blobs(n=32, n_blobs=6, sigma_range=(3, 7), seed=23)
    b = fields.grf((32, 32, 32), 3.0, seed=24)
    plan = m.Plan(dims_of(a))
    for f in (a, b, a, b):
        m.msc_compute(plan, gpu_field(f))
        off, cells = m.msc_saddle_arc_geometry(plan)
        want_off, want_cells = _want(f)
        assert np.array_equal(to_np(off), want_off)
        assert np.array_equal(to_np(cells), want_cells)
        m.msc_arc_geometry(plan)  # both geometries can be asked for in either order


@pytest.mark.slow
@pytest.mark.parametrize("name", ["grf256", "blobs512"])
def test_full_size_sampled_ss_arcs_are_single_v_paths(name):
    """The bench workloads after three passes (the replayed graph: row-wise products on the GRF, whose
    J comes from a second run of the junction waves; the junction waves on the blob field, with paths
    hundreds of cells long): sampled arcs of count 1 checked step by step against the oracle's lazily
    computed pairs."""
    m = msc()
    f = fields.config_field(name)
    d = dims_of(f)
    plan = m.Plan(d)
    dev = gpu_field(f)
    for _ in range(3):
        m.msc_compute(plan, dev)
    counts, lists = m.msc_critical(plan)
    s1, s2 = to_np(lists[1]), to_np(lists[2])
    rp, col, cnt = (to_np(x) for x in m.msc_saddle_arcs(plan))
    off, cells = m.msc_saddle_arc_geometry(plan)
    off, cells = to_np(off), to_np(cells)
    assert len(off) == len(cnt) + 1 and off[-1] == len(cells)
    assert np.all((np.diff(off) > 0) == (cnt == 1))
    rows = np.searchsorted(rp, np.arange(len(cnt)), side="right") - 1
    ones = np.nonzero(cnt == 1)[0]
    rng = np.random.default_rng(11)
    for k in rng.choice(ones, size=min(300, len(ones)), replace=False):
        path = [int(c) for c in cells[off[k]:off[k + 1]]]
        assert path[0] == int(s1[rows[k]]) and path[-1] == int(s2[col[k]])
        assert len(path) % 2 == 0 and len(set(path)) == len(path)
        pairs = oracle.lazy_pairs(f, np.array(path, np.uint32))
        assert pairs[0] == NONE and pairs[-1] == NONE  # the two saddles are critical
        for i in range(1, len(path) - 1, 2):  # quad, then the 1-cell paired with it
            assert pairs[i] == path[i + 1] and pairs[i + 1] == path[i]
        for i in range(0, len(path) - 1, 2):  # every quad is a cofacet of the 1-cell before it,
            assert pairs[i] != path[i + 1]    # other than the quad that 1-cell is paired with
            assert _is_facet(d, path[i], path[i + 1])


def _is_facet(dims, e, q):
    nx, ny, _ = dims
    rx, ry = 2 * nx - 1, 2 * ny - 1
    ec = (e % rx, (e // rx) % ry, e // (rx * ry))
    qc = (q % rx, (q // rx) % ry, q // (rx * ry))
    diff = [abs(a - b) for a, b in zip(ec, qc)]
    return sorted(diff) == [0, 0, 1] and sum(c % 2 for c in qc) == 2 and sum(c % 2 for c in ec) == 1
