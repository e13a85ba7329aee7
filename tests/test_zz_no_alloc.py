"""The no-allocation entry point msc_gradient_critical_static.

It serves callers that cannot allocate device memory: a host program that has already given
the whole GPU to its own memory pool, or code that runs inside a callback or a deadline-bound
loop where cudaMalloc is not allowed.  Its output must equal that of the regular entry points
(msc_gradient + msc_critical) bit for bit, including on consecutive calls, since every call
reuses -- and overwrites -- the same static scratch array.  This file is collected last so that
a run stopping at its first failure has run every other test first.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, run_gradient, to_np

pytestmark = pytest.mark.gpu


def _static(f):
    m = msc()
    d = gpu_field(f)
    words = torch.empty(f.shape, dtype=torch.uint32, device="cuda")
    nx, ny, nz = dims_of(f)
    capacity = [nx * ny * nz, 3 * nx * ny * nz, 3 * nx * ny * nz, nx * ny * nz]
    cells = [torch.empty(c, dtype=torch.uint32, device="cuda") for c in capacity]
    counts = m.msc_gradient_critical_static(d, words, cells, capacity)
    torch.cuda.synchronize()
    return to_np(words), counts, [to_np(cells[k][:counts[k]]) for k in range(4)]


def test_two_calls_in_a_row_match_the_regular_entry_points():
    # different shapes and fields back to back: nothing of the first call may leak into the second
    for f in (fields.grf((48, 40, 70), 3.0, seed=21), random_field((9, 8, 33), 22, "ties")):
        words, counts, lists = _static(f)
        _, want_words, want_counts, want_lists, _ = run_gradient(f)
        assert np.array_equal(words, want_words)
        assert counts == want_counts
        for k in range(4):
            assert np.array_equal(lists[k], want_lists[k])


def test_rejects_grids_beyond_the_scratch_limit_and_small_outputs():
    m = msc()
    big = torch.zeros((256, 256, 256), dtype=torch.float32, device="cuda")
    words = torch.empty((256, 256, 256), dtype=torch.uint32, device="cuda")
    cells = [torch.empty(1, dtype=torch.uint32, device="cuda") for _ in range(4)]
    with pytest.raises(m.MscError) as e:
        m.msc_gradient_critical_static(big, words, cells, [1, 1, 1, 1])
    assert e.value.status == 4  # MSC_ERR_TOO_LARGE
    f = random_field((16, 16, 16), 3)
    with pytest.raises(m.MscError) as e:
        m.msc_gradient_critical_static(gpu_field(f), torch.empty(f.shape, dtype=torch.uint32, device="cuda"),
                                       cells, [1, 1, 1, 1])
    assert e.value.status == m.MSC_ERR_CAPACITY
