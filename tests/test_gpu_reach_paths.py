"""Saddle-saddle reachability (Sec. 3.2 / 3.5) as pull sweeps over the 1-cell bitmap rows, with rows
skipped when their 3 x 3 neighbourhood did not change: the oracle's visited set and level count on
narrow, wide (rows of many words) and tiny grids, and on a few broad fronts that take many levels,
synchronised and through a replayed graph."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, edge_layout, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,f", [
    ("grf", fields.grf((64, 40, 36), 3.0, seed=71)),
    ("small", random_field((3, 5, 40), 72, "normal")),
    ("wide700", random_field((6, 20, 700), 73, "normal")),
    ("wide1300", random_field((3, 6, 1300), 74, "normal")),
    ("broad_fronts", fields.gaussian_blobs(n=48, n_blobs=3, sigma_range=(10, 16), seed=75)),
])
def test_reachability_paths(name, f):
    m = msc()
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    vis, levels = m.msc_reachability(plan)
    e = oracle.compute_all(f, with_minor=False, with_dstar=False)
    assert levels == e["levels"]
    assert np.array_equal(to_np(vis), edge_layout(e["visited"]))
    # and the same through a replayed graph
    m.msc_compute(plan, gpu_field(f))
    m.msc_compute(plan, gpu_field(f))
    vis2, levels2 = m.msc_reachability(plan)
    assert levels2 == levels and np.array_equal(to_np(vis2), to_np(vis))
