"""The no-allocation entry point msc_gradient_critical_static.

It serves callers that cannot allocate device memory: a host program that has already given
the whole GPU to its own memory pool, or code that runs inside a callback or a deadline-bound
loop where cudaMalloc is not allowed.  Its output must equal the oracle's and that of the
regular entry points (msc_gradient + msc_critical) bit for bit, including on consecutive calls,
since every call reuses -- and overwrites -- the same static scratch array.  This file is
collected last so that a run stopping at its first failure has run every other test first.
"""
from __future__ import annotations

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, run_gradient, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _outputs(f):
    d = gpu_field(f)
    words = torch.empty(f.shape, dtype=torch.uint32, device="cuda")
    nx, ny, nz = dims_of(f)
    capacity = [nx * ny * nz, 3 * nx * ny * nz, 3 * nx * ny * nz, nx * ny * nz]
    cells = [torch.empty(c, dtype=torch.uint32, device="cuda") for c in capacity]
    return d, words, cells, capacity


def _static(f):
    m = msc()
    d, words, cells, capacity = _outputs(f)
    counts = m.msc_gradient_critical_static(d, words, cells, capacity)
    torch.cuda.synchronize()
    return to_np(words), counts, [to_np(cells[k][:counts[k]]) for k in range(4)]


def test_two_calls_in_a_row_match_the_oracle_and_the_regular_entry_points():
    # different shapes and fields back to back: nothing of the first call may leak into the second
    for f in (fields.grf((48, 40, 70), 3.0, seed=21), random_field((9, 8, 33), 22, "ties")):
        words, counts, lists = _static(f)
        _, want_words, want_counts, want_lists, _ = run_gradient(f)
        assert np.array_equal(words, want_words)
        assert counts == want_counts
        for k in range(4):
            assert np.array_equal(lists[k], want_lists[k])
        pair = oracle.gradient(f)
        assert np.array_equal(words, oracle.pack(dims_of(f), pair))
        o_counts, o_lists = oracle.critical(dims_of(f), pair)
        assert counts == [int(c) for c in o_counts]
        for k in range(4):
            assert np.array_equal(lists[k], o_lists[k])


@pytest.mark.slow
def test_largest_cube_that_fits_the_scratch_and_the_first_that_does_not():
    """193^3 needs 16.70 MB of the 16 MiB scratch, 194^3 needs 16.88 MB."""
    m = msc()
    f = fields.grf((193, 193, 193), 3.0, seed=23)
    words, counts, lists = _static(f)
    _, want_words, want_counts, want_lists, _ = run_gradient(f)
    assert np.array_equal(words, want_words)
    assert counts == want_counts
    for k in range(4):
        assert np.array_equal(lists[k], want_lists[k])
    rng = np.random.default_rng(5)
    verts = rng.integers(0, f.size, size=3000)
    assert np.array_equal(words.reshape(-1)[verts], oracle.packed_at(f, verts))
    big = torch.zeros((194, 194, 194), dtype=torch.float32, device="cuda")
    out = torch.empty((194, 194, 194), dtype=torch.uint32, device="cuda")
    cells = [torch.empty(1, dtype=torch.uint32, device="cuda") for _ in range(4)]
    with pytest.raises(m.MscError) as e:
        m.msc_gradient_critical_static(big, out, cells, [1, 1, 1, 1])
    assert e.value.status == 4  # MSC_ERR_TOO_LARGE


def test_rejects_small_outputs_and_bad_buffers_before_any_launch():
    m = msc()
    f = random_field((16, 16, 16), 3)
    d, words, cells, capacity = _outputs(f)
    small = [torch.empty(1, dtype=torch.uint32, device="cuda") for _ in range(4)]
    with pytest.raises(m.MscError) as e:
        m.msc_gradient_critical_static(d, words, small, [1, 1, 1, 1])
    assert e.value.status == m.MSC_ERR_CAPACITY
    # a capacity beyond the tensor would let the kernel write past its end: refused on the host
    with pytest.raises(ValueError):
        m.msc_gradient_critical_static(d, words, small, [1, 1, 1, 2])
    with pytest.raises(ValueError):
        m.msc_gradient_critical_static(d, words, [c.view(torch.int32) for c in cells], capacity)
    with pytest.raises(ValueError):
        m.msc_gradient_critical_static(d, words, [c.cpu() for c in cells], capacity)
    with pytest.raises(ValueError):
        m.msc_gradient_critical_static(d, words.view(torch.int32), cells, capacity)


_RESERVED_RUN = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2009_03707_gb300 import msc
from synth import fields
torch.cuda.set_device(0)
f = fields.grf((40, 44, 37), 3.0, seed=31)
d = torch.from_numpy(f).cuda()
nz, ny, nx = f.shape
plan = msc.Plan((nx, ny, nz))
msc.msc_gradient(plan, d)
counts, cells = msc.msc_critical(plan)
want = (msc.msc_gradient_words(plan).cpu(), counts, [c.cpu() for c in cells])
del plan, cells
words = torch.empty(f.shape, dtype=torch.uint32, device="cuda")
cap = [f.size, 3 * f.size, 3 * f.size, f.size]
out = [torch.empty(c, dtype=torch.uint32, device="cuda") for c in cap]
torch.cuda.synchronize()
msc.msc_static_prepare(0)
# hold all but a few MB of the device, as a host program with its own pool would (a block of
# exactly "free" bytes may not exist, so the margin grows until one allocation succeeds)
free, _ = torch.cuda.mem_get_info()
hold = None
for margin in (16, 32, 64, 128, 256, 512):
    try:
        hold = torch.empty(free - (margin << 20), dtype=torch.uint8, device="cuda")
        break
    except Exception:
        torch.cuda.empty_cache()
assert hold is not None
for _ in range(2):  # compared on the host: any device-side op would need memory of its own
    got = msc.msc_gradient_critical_static(d, words, out, cap)
    torch.cuda.synchronize()
    assert got == want[1], (got, want[1])
    assert torch.equal(words.cpu(), want[0])
    for k in range(4):
        assert torch.equal(out[k][:got[k]].cpu(), want[2][k])
left, _ = torch.cuda.mem_get_info()
print("ok", left >> 20)
"""


def test_prepared_device_runs_with_its_memory_reserved():
    """In a fresh process: prepare the device, then take all but a few MB of its memory for
    ourselves (as a host program with its own pool would) and run the entry point twice."""
    r = subprocess.run([sys.executable, "-c", _RESERVED_RUN, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.startswith("ok")
