"""Bit-exact parity of the batching and serving runtime on its two workloads as configured:

* the uneven batch: 64 Gaussian random fields (P(k) ~ k^-2.5, seeds 100-163), each axis drawn in
  48..192, submitted as one batch -- the first submission (one job per volume) and the group
  graph's replay (one launch for all 64);
* the serving stream: all 8 advected fields (cubes of 64..384), two time steps each, through
  msc_batch_submit with each stream's plan reused across its steps, under an 8 GiB admission
  budget.

The oracle cannot run 112 M voxels whole in test time (about 0.12 Mvoxel/s), so every volume's
outputs are checked at sampled vertices, cubes and 1-saddles against its lazy queries (lower stars
computed one at a time), every volume's critical counts against the Euler characteristic and the
zero codes of its words, and the smallest volumes' counts against the whole-volume oracle, run in
a process pool started before any GPU work.  Every request must also equal the same volume run
alone."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from synth import fields
from tests import oracle_pool
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _outputs(m, plan):
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    rp, col, cnt = m.msc_saddle_arcs(plan)
    return dict(words=to_np(m.msc_gradient_words(plan)), counts=counts, cells=[to_np(c) for c in cells],
                amin=to_np(amin), amax=to_np(amax), vmin=to_np(vmin).reshape(-1), cmax=to_np(cmax).reshape(-1),
                rowptr=to_np(rp), col=to_np(col), cnt=to_np(cnt))


def _same(a, b):
    assert a["counts"] == b["counts"]
    for k in range(4):
        assert np.array_equal(a["cells"][k], b["cells"][k])
    for key in ("words", "amin", "amax", "vmin", "cmax", "rowptr", "col", "cnt"):
        assert np.array_equal(a[key], b[key]), key


def _check_sampled(f, r, rng, n_verts, n_rows):
    """Sampled outputs of one volume against the lazy oracle, and count properties."""
    nz, ny, nx = f.shape
    rx, ry = 2 * nx - 1, 2 * ny - 1
    counts = r["counts"]
    assert counts[0] - counts[1] + counts[2] - counts[3] == 1
    flat = r["words"].reshape(-1)
    assert sum(int((((flat >> np.uint32(3 * s)) & 7) == 0).sum()) for s in range(8)) == sum(counts)
    v = rng.integers(0, f.size, size=n_verts)
    assert np.array_equal(flat[v], oracle.packed_at(f, v))
    assert np.array_equal(r["vmin"][v], oracle.lazy_vertex_min(f, v))
    assert np.array_equal(r["cmax"][v], oracle.lazy_cube_max(f, v))
    i1 = rng.integers(0, counts[1], size=min(counts[1], n_rows))
    e = r["cells"][1][i1].astype(np.int64)
    ex, ey, ez = e % rx, (e // rx) % ry, e // (rx * ry)
    lo = (ex // 2) + nx * ((ey // 2) + ny * (ez // 2))
    assert np.array_equal(r["amin"][2 * i1], oracle.lazy_vertex_min(f, lo))
    rows = np.unique(i1)
    want = oracle.lazy_dstar_rows(f, r["cells"][1][rows])
    rp = r["rowptr"]
    for s in rows:
        a, b = int(rp[s]), int(rp[s + 1])
        got = {int(r["cells"][2][c]): int(k) for c, k in zip(r["col"][a:b], r["cnt"][a:b])}
        assert got == want[int(r["cells"][1][s])]


def _pool():
    return cf.ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=mp.get_context("spawn"))


def test_uneven_batch_of_64_as_configured():
    vols = fields.batch_volumes(64)
    sizes = np.array([f.size for f in vols])
    small = [int(i) for i in np.argsort(sizes)[:12]]
    with _pool() as pool:  # started before the first GPU call of this test
        futs = {i: pool.submit(oracle_pool.critical_counts, vols[i]) for i in small}
        m = msc()
        dev = [gpu_field(f) for f in vols]
        batch = m.Batch(n_workers=4)
        ticket, plans = batch.msc_batch_submit(dev)  # first run of every plan: one job per volume
        assert batch.msc_batch_wait(ticket) == 0
        first = [_outputs(m, p) for p in plans]
        for _ in range(2):  # the group graph: captured, then replayed
            ticket, _ = batch.msc_batch_submit(dev, plans)
            assert batch.msc_batch_wait(ticket) == 0
        replay = [_outputs(m, p) for p in plans]
        rng = np.random.default_rng(64)
        for i, f in enumerate(vols):
            _same(replay[i], first[i])
            _check_sampled(f, replay[i], rng, n_verts=400, n_rows=12)
        for i in small:
            assert replay[i]["counts"] == futs[i].result(), i
        # a few volumes alone, on fresh plans
        for i in (0, int(np.argmax(sizes)), small[0]):
            alone = m.Plan(dims_of(vols[i]))
            m.msc_compute(alone, dev[i])
            _same(_outputs(m, alone), replay[i])
        batch.close()


def test_serving_streams_as_configured():
    m = msc()
    streams = fields.serving_streams()
    assert [s.size for s in streams] == [64, 110, 155, 201, 247, 293, 338, 384]
    batch = m.Batch(n_workers=4, hbm_budget_bytes=8 << 30)
    plans = [None] * len(streams)
    rng = np.random.default_rng(500)
    for t in range(2):
        steps = [s.step_device(t) for s in streams]
        ticket, plans = batch.msc_batch_submit(steps, plans)  # each stream keeps its plan
        assert batch.msc_batch_wait(ticket) == 0
        for s, d, plan in zip(streams, steps, plans):
            got = _outputs(m, plan)
            alone = m.Plan((s.size,) * 3)
            m.msc_compute(alone, d)
            _same(got, _outputs(m, alone))
            del alone
            _check_sampled(d.cpu().numpy(), got, rng, n_verts=300, n_rows=8)
        del steps
    batch.close()
