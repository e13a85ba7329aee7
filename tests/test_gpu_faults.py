"""Failure detection without a GPU fault: failures are made on the host (a faked allocation
failure, a status bit raised the way a bounded wait or an overflow check raises it, an iteration
cap that trips) and every call must return a clean status, leave the process usable, and in a
batch fail only the volume it hits.  Each case runs in a child process so that MSC_FAULT is read
fresh at plan creation."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2009_03707_gb300 import msc
from synth import fields
f = torch.from_numpy(fields.grf((24, 26, 28), 3.0, seed=3)).cuda()
try:
    plan = msc.Plan((28, 26, 24), max_iterations={maxit})
    msc.msc_compute(plan, f)
    print("STATUS 0")
except msc.MscError as e:
    print("STATUS", e.status, str(e))
# the process stays usable: a fresh plan without the fault completes
import os; os.environ.pop("MSC_FAULT", None)
ok = msc.Plan((28, 26, 24))
msc.msc_compute(ok, f)
print("AFTER", msc.msc_get_stats(ok)["counts"])
"""


def _child(fault, maxit=0):
    env = dict(os.environ)
    if fault:
        env["MSC_FAULT"] = fault
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, maxit=maxit)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = dict(l.split(" ", 1) for l in r.stdout.splitlines() if " " in l)
    return int(lines["STATUS"].split()[0]), lines


@pytest.mark.parametrize("fault,status", [("alloc@1", 3), ("alloc@7", 3), ("timeout", 8), ("overflow", 6), (None, 0)])
def test_injected_faults_return_clean_status(fault, status):
    st, lines = _child(fault)
    assert st == status, lines
    assert lines["AFTER"].startswith("[")


def test_iteration_cap_trips_cleanly():
    st, lines = _child(None, maxit=1)
    assert st == 7, lines  # MSC_ERR_ITER_LIMIT


def test_batch_isolates_a_failing_volume(monkeypatch):
    """One volume of a batch fails (NaN); the others complete with correct results."""
    import numpy as np
    import torch

    from tests.gpu_util import gpu_field, msc, to_np
    from tests.cubical import random_field

    m = msc()
    good = [random_field((10, 11, 12), i) for i in range(4)]
    bad = random_field((10, 11, 12), 9)
    bad[3, 3, 3] = np.nan
    batch = m.Batch(n_workers=3)
    ticket, plans = batch.msc_batch_submit([gpu_field(x) for x in good[:2] + [bad] + good[2:]])
    assert batch.msc_batch_wait(ticket) == 2
    for f, plan in zip(good, plans[:2] + plans[3:]):
        alone = m.Plan((12, 11, 10))
        m.msc_compute(alone, gpu_field(f))
        assert m.msc_critical(plan)[0] == m.msc_critical(alone)[0]
        assert np.array_equal(to_np(m.msc_saddle_arcs(plan)[2]), to_np(m.msc_saddle_arcs(alone)[2]))
    batch.close()
