"""Arc geometry (the cells along every saddle-extremum arc, Sec. 3.4 / Sec. 3.5 "Data structure"):
msc_arc_geometry and msc_copy_to_host against the oracle's walks, element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


def _cases():
    out = [("cos32", fields.cosine_lattice()), ("grf40", fields.grf((40, 36, 44), 3.0, seed=12)),
           ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5))]
    for i, shp in enumerate([(2, 2, 2), (3, 5, 7), (9, 8, 33), (17, 16, 65), (64, 2, 3), (2, 30, 2)]):
        out.append((f"normal{shp}", random_field(shp, 900 + i, "normal")))
        out.append((f"ties{shp}", random_field(shp, 950 + i, "ties")))
    return out


def _want(f):
    d = dims_of(f)
    pair = oracle.gradient(f)
    _, lists = oracle.critical(d, pair)
    return oracle.arc_cells(d, pair, lists[1], lists[2])


@pytest.mark.parametrize("name,f", _cases(), ids=[n for n, _ in _cases()])
def test_arc_geometry_matches_oracle(name, f):
    m = msc()
    plan = m.Plan(dims_of(f))
    m.msc_gradient(plan, gpu_field(f))  # the geometry needs only the gradient and the critical cells
    off, cells = m.msc_arc_geometry(plan)
    want_off, want_cells = _want(f)
    assert np.array_equal(to_np(off), want_off)
    assert np.array_equal(to_np(cells), want_cells)
    assert np.array_equal(m.msc_copy_to_host(plan, "arc_offsets"), want_off)
    assert np.array_equal(m.msc_copy_to_host(plan, "arc_cells"), want_cells)


def test_geometry_of_replayed_passes_follows_the_field():
    """Built once per pass and dropped by the next: after replays of two fields on one plan, each
    query returns the current field's arcs."""
    m = msc()
    a = fields.grf((30, 33, 28), 3.0, seed=41)
    b = random_field((30, 33, 28), 42, "normal")
    plan = m.Plan(dims_of(a))
    for f in (a, b, a, b):
        m.msc_compute(plan, gpu_field(f))
        off, cells = m.msc_arc_geometry(plan)
        want_off, want_cells = _want(f)
        assert np.array_equal(to_np(off), want_off)
        assert np.array_equal(to_np(cells), want_cells)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["grf256", "blobs512"])
def test_full_size_sampled_arcs_are_v_paths(name):
    """The bench workloads after three passes (the replayed graph): sampled arcs checked cell by cell
    against the oracle's lazily computed pairs, ending at the pass's arc end points."""
    m = msc()
    f = fields.config_field(name)
    plan = m.Plan(dims_of(f))
    d = gpu_field(f)
    for _ in range(3):
        m.msc_compute(plan, d)
    counts, lists = m.msc_critical(plan)
    amin, amax, _, _ = m.msc_extremum_arcs(plan)
    amin, amax = to_np(amin), to_np(amax)
    off, cells = m.msc_arc_geometry(plan)
    off, cells = to_np(off), to_np(cells)
    n1, n2 = counts[1], counts[2]
    assert len(off) == 2 * (n1 + n2) + 1 and off[-1] == len(cells)
    rng = np.random.default_rng(7)
    picks = np.concatenate([rng.integers(0, 2 * n1, 150), 2 * n1 + rng.integers(0, 2 * n2, 150)])
    for a in picks:
        path = cells[off[a]:off[a + 1]]
        pairs = oracle.lazy_pairs(f, path)
        # consecutive cells are pairs or facet steps: every second step is a gradient pair
        for k in range(1, len(path) - 1, 2):
            assert pairs[k] == path[k + 1]
        if a < 2 * n1:
            assert pairs[-1] == NONE and path[-1] == amin[a]
        else:
            b = a - 2 * n1
            if pairs[-1] == NONE and len(path) > 1 and len(path) % 2 == 0:
                assert path[-1] == amax[b]  # ended at a maximum
            else:
                assert amax[b] == NONE  # left the domain, or no cube on that side
