"""The 1-skeleton adjacency exported to the host (msc_complex_graph: every arc at both ends,
Sec. 3.5 "Data structure").  Small fields: equal to the oracle's adjacency built from the oracle's
arcs.  Larger fields (multi-pass sorts): equal to the same plain construction applied to the
library's own arc outputs, which the pipeline tests pin to the oracle.  Also the size query and
the capacity error of the C ABI."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _run(m, f):
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    return plan


def _same(got, want):
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g), np.asarray(w))


@pytest.mark.parametrize("name,f", [
    ("cos32", fields.cosine_lattice()),
    ("grf40", fields.grf((40, 40, 40), 3.0, seed=21)),
    ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5)),
    ("normal9x8x33", random_field((9, 8, 33), 31, "normal")),
    ("ties6", random_field((6, 6, 6), 32, "ties")),
    ("tiny2", random_field((2, 2, 2), 33, "normal")),
])
def test_graph_matches_oracle(name, f):
    m = msc()
    plan = _run(m, f)
    e = oracle.compute_all(f, with_minor=False, with_dstar=True)
    want = oracle.complex_graph(e["counts"], e["lists"], e["min_arcs"], e["max_arcs"], e["dstar"])
    _same(m.msc_complex_graph(plan), want)


@pytest.mark.parametrize("shape,alpha,seed", [((72, 64, 60), 2.0, 3), ((128, 128, 96), 2.5, 4)])
def test_graph_from_library_arcs(shape, alpha, seed):
    m = msc()
    f = fields.grf(shape, alpha, seed=seed)
    plan = _run(m, f)
    counts, cells = m.msc_critical(plan)
    amin, amax, _, _ = m.msc_extremum_arcs(plan)
    rowptr, col, cnt = (to_np(x) for x in m.msc_saddle_arcs(plan))
    rows = np.repeat(np.arange(len(rowptr) - 1, dtype=np.uint32), np.diff(rowptr))
    want = oracle.complex_graph(counts, [to_np(c) for c in cells], to_np(amin), to_np(amax), (rows, col, cnt))
    _same(m.msc_complex_graph(plan), want)


def test_size_query_and_capacity():
    m = msc()
    f = fields.grf((30, 30, 30), 3.0, seed=9)
    plan = _run(m, f)
    lib = m.lib
    n_nodes, n_adj = ctypes.c_int64(), ctypes.c_int64(0)
    assert lib.msc_complex_graph(plan.handle, None, ctypes.byref(n_nodes), ctypes.byref(n_adj), None, None, None) == 0
    counts, _ = m.msc_critical(plan)
    assert n_nodes.value == sum(int(c) for c in counts) and n_adj.value > 0
    nodeptr = np.zeros(n_nodes.value + 1, np.int64)
    adj = np.zeros(n_adj.value, np.uint32)
    mult = np.zeros(n_adj.value, np.uint64)
    small = ctypes.c_int64(n_adj.value - 1)
    args = [nodeptr.ctypes.data_as(ctypes.c_void_p), adj.ctypes.data_as(ctypes.c_void_p),
            mult.ctypes.data_as(ctypes.c_void_p)]
    assert lib.msc_complex_graph(plan.handle, None, ctypes.byref(n_nodes), ctypes.byref(small), *args) == 12
    assert small.value == n_adj.value and not nodeptr.any()   # sizes reported, nothing copied
    full = ctypes.c_int64(n_adj.value)
    assert lib.msc_complex_graph(plan.handle, None, ctypes.byref(n_nodes), ctypes.byref(full), *args) == 0
    assert nodeptr[-1] == n_adj.value
