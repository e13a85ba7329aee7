"""msc_compute_async / msc_compute_wait: a pass enqueued without waiting, on the plan's graph.
Every output must equal a synchronised run's (MSC_FLAG_NO_GRAPH), with two plans' passes in flight
on two streams, when a query arrives before the wait, when a pass fails (NaN), and when a pass
outgrows the captured capacities (it is re-run synchronised inside the wait)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _outputs(m, plan):
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    rowptr, col, cnt = m.msc_saddle_arcs(plan)
    return [np.asarray(counts)] + [to_np(c) for c in cells] + [to_np(x) for x in (amin, amax, vmin, cmax, rowptr, col, cnt)]


def _reference(m, f):
    plan = m.Plan(dims_of(f), no_graph=True)
    m.msc_compute(plan, gpu_field(f))
    return _outputs(m, plan)


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_two_plans_in_flight():
    m = msc()
    shape = (36, 40, 33)
    fs = [fields.grf(shape, 3.0, seed=s) for s in (51, 52, 53, 54)]
    want = [_reference(m, f) for f in fs]
    plans = [m.Plan(dims_of(fs[0])) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    bufs = [gpu_field(fs[0]), gpu_field(fs[0])]
    for x in range(2):  # first (synchronised) runs, then the graphs are captured by the async calls
        with torch.cuda.stream(streams[x]):
            m.msc_compute(plans[x], bufs[x])
    for rep in range(2):
        for i, f in enumerate(fs):
            x = i % 2
            with torch.cuda.stream(streams[x]):
                m.msc_compute_wait(plans[x])          # the previous pass on this plan
                bufs[x].copy_(gpu_field(f))
                m.msc_compute_async(plans[x], bufs[x])
            y = 1 - x
            if i > 0:
                with torch.cuda.stream(streams[y]):
                    m.msc_compute_wait(plans[y])
                    _same(_outputs(m, plans[y]), want[i - 1])
        with torch.cuda.stream(streams[(len(fs) - 1) % 2]):
            m.msc_compute_wait(plans[(len(fs) - 1) % 2])
            _same(_outputs(m, plans[(len(fs) - 1) % 2]), want[-1])


def test_query_before_wait_waits():
    m = msc()
    f = fields.grf((30, 31, 32), 3.0, seed=61)
    plan = m.Plan(dims_of(f))
    buf = gpu_field(f)
    m.msc_compute(plan, buf)
    m.msc_compute_async(plan, buf)
    _same(_outputs(m, plan), _reference(m, f))   # no explicit wait
    st = m.msc_get_stats(plan)
    assert st["n_junctions"] > 0
    m.msc_compute_wait(plan)                      # nothing in flight: returns at once


def test_error_reported_by_wait():
    m = msc()
    f = fields.grf((20, 21, 22), 3.0, seed=62)
    plan = m.Plan(dims_of(f))
    buf = gpu_field(f)
    for _ in range(2):
        m.msc_compute(plan, buf)
    bad = f.copy()
    bad[3, 4, 5] = np.nan
    buf.copy_(gpu_field(bad))
    m.msc_compute_async(plan, buf)
    with pytest.raises(m.MscError) as e:
        m.msc_compute_wait(plan)
    assert e.value.status == 2
    buf.copy_(gpu_field(f))
    m.msc_compute_async(plan, buf)
    m.msc_compute_wait(plan)
    _same(_outputs(m, plan), _reference(m, f))


def test_capacity_overflow_in_wait():
    m = msc()
    smooth = fields.grf((34, 34, 34), 4.5, seed=63)
    rough = random_field((34, 34, 34), 64, "normal")
    plan = m.Plan(dims_of(smooth))
    buf = gpu_field(smooth)
    for _ in range(2):
        m.msc_compute(plan, buf)
    buf.copy_(gpu_field(rough))
    m.msc_compute_async(plan, buf)
    m.msc_compute_wait(plan)
    _same(_outputs(m, plan), _reference(m, rough))
    m.msc_compute_async(plan, buf)   # re-captured with the larger capacities
    m.msc_compute_wait(plan)
    _same(_outputs(m, plan), _reference(m, rough))
