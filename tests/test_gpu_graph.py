"""msc_compute replays the whole pipeline as one captured CUDA graph after its first call on a
plan.  Every output of a replay must equal the synchronised run's (MSC_FLAG_NO_GRAPH) and the
oracle's, including when the field changes under the same plan, when a new field needs more room
than the graph was captured with (the pass is rerun and the graph re-captured), and for a new
field pointer."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _outputs(m, plan):
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    vis, levels = m.msc_reachability(plan)
    out = dict(counts=list(counts), cells=[to_np(c) for c in cells], amin=to_np(amin), amax=to_np(amax),
               vmin=to_np(vmin), cmax=to_np(cmax), visited=to_np(vis), levels=levels,
               junctions=to_np(m.msc_junctions(plan)),
               minor=[tuple(to_np(x) for x in m.msc_minor(plan, w)) for w in range(4)],
               dstar=tuple(to_np(x) for x in m.msc_saddle_arcs(plan)))
    st = m.msc_get_stats(plan)
    # (left out: the pointer-jumping round count -- in-place jumping may finish a round early,
    # depending on thread scheduling -- and the path-count work count, whose meaning depends on
    # the method a run used; the outputs depend on neither)
    out["stats"] = {k: st[k] for k in ("n_reachable", "n_bfs_levels", "n_junctions", "nnz_A", "nnz_B", "nnz_Bstar",
                                       "nnz_D", "nnz_Dstar", "n_iter", "max_path_count")}
    return out


def _assert_same(a, b):
    for key in a:
        if key in ("cells", "minor", "dstar"):
            for x, y in zip(a[key], b[key]):
                if isinstance(x, tuple):
                    for u, v in zip(x, y):
                        assert np.array_equal(u, v), key
                else:
                    assert np.array_equal(x, y), key
        elif isinstance(a[key], np.ndarray):
            assert np.array_equal(a[key], b[key]), key
        else:
            assert a[key] == b[key], key


def _reference(m, f):
    plan = m.Plan(dims_of(f), no_graph=True)
    m.msc_compute(plan, gpu_field(f))
    return _outputs(m, plan)


@pytest.mark.parametrize("serial", [False, True])
@pytest.mark.parametrize("shape,alpha,seed", [((40, 40, 40), 3.0, 1), ((33, 20, 47), 2.5, 2)])
def test_replays_match_synchronised_runs(shape, alpha, seed, serial):
    """Replays with the saddle-extremum stage on its own branch (the default) and as one chain
    (MSC_FLAG_SERIAL_PASS)."""
    m = msc()
    fa = fields.grf(shape, alpha, seed=seed)
    fb = fields.grf(shape, alpha, seed=seed + 100)
    plan = m.Plan(dims_of(fa), serial_pass=serial)
    da = gpu_field(fa)
    want_a, want_b = _reference(m, fa), _reference(m, fb)
    for _ in range(3):  # synchronised run, then capture + replay, then replay
        m.msc_compute(plan, da)
        _assert_same(_outputs(m, plan), want_a)
    db = gpu_field(fb)  # a new pointer: captured anew
    for _ in range(2):
        m.msc_compute(plan, db)
        _assert_same(_outputs(m, plan), want_b)
    # the same buffer refilled with field a: the replay reads the new contents
    db.copy_(da)
    m.msc_compute(plan, db)
    _assert_same(_outputs(m, plan), want_a)


def test_capacity_overflow_reruns_and_recaptures():
    """A smooth field sets small capacities; a rough one on the same plan outgrows them."""
    m = msc()
    smooth = fields.grf((36, 36, 36), 4.5, seed=7)
    rough = random_field((36, 36, 36), 8, "normal")
    plan = m.Plan(dims_of(smooth))
    buf = gpu_field(smooth)
    for _ in range(2):
        m.msc_compute(plan, buf)
    buf.copy_(gpu_field(rough))
    want = _reference(m, rough)
    for _ in range(3):
        m.msc_compute(plan, buf)
        _assert_same(_outputs(m, plan), want)
    e = oracle.compute_all(rough, with_minor=False, with_dstar=True)
    got = _outputs(m, plan)
    assert got["counts"] == [int(c) for c in e["counts"]]
    rows, cols, cnt = e["dstar"]
    rowptr, col, count = got["dstar"]
    assert np.array_equal(col, cols) and np.array_equal(count, cnt)


def test_replay_reports_errors():
    """A NaN in a replayed field is reported like in a synchronised run, and the plan recovers."""
    m = msc()
    f = fields.grf((20, 21, 22), 3.0, seed=4)
    plan = m.Plan(dims_of(f))
    buf = gpu_field(f)
    for _ in range(2):
        m.msc_compute(plan, buf)
    bad = f.copy()
    bad[5, 6, 7] = np.nan
    buf.copy_(gpu_field(bad))
    with pytest.raises(m.MscError) as e:
        m.msc_compute(plan, buf)
    assert e.value.status == 2
    buf.copy_(gpu_field(f))
    m.msc_compute(plan, buf)
    _assert_same(_outputs(m, plan), _reference(m, f))


@pytest.mark.parametrize("method", [1, 2])
def test_replays_with_each_path_count_method(method):
    """Graph replays run the path count as row-wise products or as junction waves (a WHILE loop of
    waves); both give the oracle's D* on a field with a deep minor."""
    m = msc()
    f = fields.gaussian_blobs(n=40, n_blobs=5, sigma_range=(4, 12), seed=11)
    e = oracle.compute_all(f, with_minor=True, with_dstar=True)
    plan = m.Plan(dims_of(f), path_count_method=method)
    buf = gpu_field(f)
    for _ in range(3):
        m.msc_compute(plan, buf)
        rowptr, col, cnt = (to_np(x) for x in m.msc_saddle_arcs(plan))
        er, ec, en = e["dstar"]
        assert np.array_equal(col, ec) and np.array_equal(cnt, en)
        assert np.array_equal(np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr)), er)
        st = m.msc_get_stats(plan)
        assert st["n_iter"] == e["n_iter"] and st["path_count_method"] == method
