"""Batching and serving runtime (msc_batch_submit / msc_poll): volumes of uneven size run
concurrently on worker streams; every result must equal the one computed alone (and the
oracle), whatever the mix, the admission budget or the reuse of a plan across time steps."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import csr_to_coo, dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _outputs(m, plan):
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    rp, col, cnt = m.msc_saddle_arcs(plan)
    return dict(counts=counts, cells=[to_np(c) for c in cells], amin=to_np(amin), amax=to_np(amax),
                vmin=to_np(vmin), cmax=to_np(cmax), dstar=csr_to_coo(to_np(rp), to_np(col), to_np(cnt)))


def _alone(m, f):
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    return _outputs(m, plan)


def _same(a, b):
    assert a["counts"] == b["counts"]
    for k in range(4):
        assert np.array_equal(a["cells"][k], b["cells"][k])
    for key in ("amin", "amax", "vmin", "cmax"):
        assert np.array_equal(a[key], b[key]), key
    for x, y in zip(a["dstar"], b["dstar"]):
        assert np.array_equal(x, y)


def _volumes():
    vols = [fields.batch_volume(100 + i, lo=12, hi=40) for i in range(6)]
    vols.append(random_field((7, 9, 33), 5, "ties"))
    return vols


@pytest.mark.parametrize("workers,budget", [(3, 0), (4, 1 << 20), (1, 0)])
def test_batch_results_equal_alone_and_oracle(workers, budget):
    m = msc()
    vols = _volumes()
    batch = m.Batch(n_workers=workers, hbm_budget_bytes=budget)
    dev = [gpu_field(f) for f in vols]
    ticket, plans = batch.msc_batch_submit(dev)
    assert batch.msc_batch_wait(ticket) == 0
    done, status = batch.msc_poll(ticket)
    assert done and status == 0
    for f, plan in zip(vols, plans):
        got = _outputs(m, plan)
        _same(got, _alone(m, f))
        e = oracle.compute_all(f)
        assert np.array_equal(csr_to_coo(*[to_np(x) for x in m.msc_saddle_arcs(plan)])[2], e["dstar"][2])
        assert got["counts"] == [int(c) for c in e["counts"]]
    batch.close()


def test_plan_reuse_across_time_steps_and_poll_does_not_block():
    m = msc()
    base = fields.serving_streams(n_streams=2, lo=20, hi=28)
    batch = m.Batch(n_workers=2)
    plans = [None, None]
    tickets = []
    for t in range(3):
        steps = [gpu_field(s.step(t)) for s in base]
        ticket, plans = batch.msc_batch_submit(steps, plans)  # the same two plans every step
        t0 = time.perf_counter()
        batch.msc_poll(ticket)
        assert time.perf_counter() - t0 < 0.05
        tickets.append((ticket, [s.step(t) for s in base]))
        assert batch.msc_batch_wait(ticket) == 0
        for plan, f in zip(plans, tickets[-1][1]):
            _same(_outputs(m, plan), _alone(m, f))
    batch.close()


def test_batch_reports_errors_per_ticket():
    m = msc()
    bad = random_field((8, 8, 8), 1)
    bad[2, 3, 4] = np.nan
    batch = m.Batch(n_workers=2)
    ticket, _ = batch.msc_batch_submit([gpu_field(random_field((8, 8, 8), 2)), gpu_field(bad)])
    assert batch.msc_batch_wait(ticket) == 2  # MSC_ERR_NAN
    batch.close()


def test_group_graph_replays_equal_alone():
    """Once every plan of a submission has run, the submission runs as one graph with a branch per
    volume; its replays (same plans, same buffers, new contents) must give each volume's own
    results."""
    m = msc()
    vols = _volumes()
    dev = [gpu_field(f) for f in vols]
    batch = m.Batch(n_workers=2)
    ticket, plans = batch.msc_batch_submit(dev)  # first run of every plan: one job per volume
    assert batch.msc_batch_wait(ticket) == 0
    for rnd in range(3):  # group capture, then replays
        if rnd == 2:  # new contents in the same buffers
            vols = [np.ascontiguousarray(np.roll(f, 3, axis=0)) for f in vols]
            for d, f in zip(dev, vols):
                d.copy_(gpu_field(f))
        ticket, _ = batch.msc_batch_submit(dev, plans)
        assert batch.msc_batch_wait(ticket) == 0
        for f, plan in zip(vols, plans):
            _same(_outputs(m, plan), _alone(m, f))
    batch.close()


def test_group_volume_outgrowing_its_branch_is_rerun():
    m = msc()
    smooth = [fields.grf((30, 28, 26), 4.5, seed=20 + i) for i in range(3)]
    dev = [gpu_field(f) for f in smooth]
    batch = m.Batch(n_workers=2)
    ticket, plans = batch.msc_batch_submit(dev)
    assert batch.msc_batch_wait(ticket) == 0
    ticket, _ = batch.msc_batch_submit(dev, plans)  # captured with the smooth fields' sizes
    assert batch.msc_batch_wait(ticket) == 0
    rough = random_field((30, 28, 26), 31, "normal")
    dev[1].copy_(gpu_field(rough))
    for _ in range(2):
        ticket, _ = batch.msc_batch_submit(dev, plans)
        assert batch.msc_batch_wait(ticket) == 0
        for f, plan in zip([smooth[0], rough, smooth[2]], plans):
            _same(_outputs(m, plan), _alone(m, f))
    batch.close()


def test_on_request_outputs_of_batch_plans_equal_alone():
    """The on-request outputs -- both arc geometries, the host 1-skeleton and a simplification -- of
    the plans a batch submission returns equal those of the same volumes computed alone, after the
    first submission and after the group graph's replay."""
    m = msc()
    vols = _volumes()[:4] + [fields.gaussian_blobs(n=28, n_blobs=5, sigma_range=(3, 7), seed=71)]
    batch = m.Batch(n_workers=3)
    dev = [gpu_field(f) for f in vols]
    ticket, plans = batch.msc_batch_submit(dev)
    assert batch.msc_batch_wait(ticket) == 0
    for rep in range(2):
        if rep:
            ticket, _ = batch.msc_batch_submit(dev, plans)
            assert batch.msc_batch_wait(ticket) == 0
        for f, d, plan in zip(vols, dev, plans):
            alone = m.Plan(dims_of(f))
            m.msc_compute(alone, d)
            for fn in (m.msc_arc_geometry, m.msc_saddle_arc_geometry):
                for x, y in zip(fn(plan), fn(alone)):
                    assert np.array_equal(to_np(x), to_np(y)), fn.__name__
            for x, y in zip(m.msc_complex_graph(plan), m.msc_complex_graph(alone)):
                assert np.array_equal(x, y)
            thr = 0.1 * float(f.max() - f.min())
            a, b = m.msc_simplify(plan, d, thr), m.msc_simplify(alone, d, thr)
            assert a["counts"] == b["counts"] and a["n_rounds"] == b["n_rounds"]
            for key in ("alive", "nodeptr", "adj", "mult", "log"):
                assert np.array_equal(to_np(a[key]), to_np(b[key])), key
    batch.close()
