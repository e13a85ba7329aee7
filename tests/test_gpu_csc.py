"""The saddle-saddle arcs by 2-saddle (the compressed sparse column form of D*, Sec. 3.5 "Data
structure": every arc is stored in both directions).  Small fields: element by element against
the oracle's D* sorted by (2-saddle, 1-saddle).  Larger fields, where the sort takes two and three
digit passes: against the transpose of the library's own CSR, which the pipeline tests pin to the
oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _csc(m, f):
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    counts, _ = m.msc_critical(plan)
    csr = tuple(to_np(x) for x in m.msc_saddle_arcs(plan))
    csc = tuple(to_np(x) for x in m.msc_saddle_arcs_csc(plan))
    return counts, csr, csc


def _transpose(n2, rowptr, col, cnt):
    rows = np.repeat(np.arange(len(rowptr) - 1, dtype=np.int64), np.diff(rowptr))
    order = np.lexsort((rows, col.astype(np.int64)))
    colptr = np.zeros(n2 + 1, dtype=np.int64)
    np.add.at(colptr, col.astype(np.int64) + 1, 1)
    return np.cumsum(colptr), rows[order].astype(np.uint32), cnt[order]


@pytest.mark.parametrize("name,f", [
    ("cos32", fields.cosine_lattice()),
    ("grf40", fields.grf((40, 40, 40), 3.0, seed=21)),
    ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5)),
    ("normal9x8x33", random_field((9, 8, 33), 31, "normal")),
    ("ties6", random_field((6, 6, 6), 32, "ties")),
    ("tiny2", random_field((2, 2, 2), 33, "normal")),
])
def test_csc_matches_oracle(name, f):
    m = msc()
    counts, _, (colptr, row, cnt) = _csc(m, f)
    e = oracle.compute_all(f, with_minor=False, with_dstar=True)
    er, ec, en = e["dstar"]
    order = np.lexsort((er.astype(np.int64), ec.astype(np.int64)))
    n2 = int(e["counts"][2])
    assert len(colptr) == n2 + 1 and colptr[0] == 0 and colptr[-1] == len(er)
    assert np.array_equal(np.diff(colptr), np.bincount(ec.astype(np.int64), minlength=n2))
    assert np.array_equal(row, er[order]) and np.array_equal(cnt, en[order])


@pytest.mark.parametrize("shape,alpha,seed", [((72, 64, 60), 2.0, 3), ((128, 128, 96), 2.5, 4)])
def test_csc_is_the_transpose(shape, alpha, seed):
    """Enough 2-saddles for two (> 256) and three (> 65536) digit passes of the column sort."""
    m = msc()
    f = fields.grf(shape, alpha, seed=seed)
    counts, (rowptr, col, cnt), (colptr, row, ccnt) = _csc(m, f)
    n2 = int(counts[2])
    assert n2 > 256
    want = _transpose(n2, rowptr, col, cnt)
    assert np.array_equal(colptr, want[0])
    assert np.array_equal(row, want[1]) and np.array_equal(ccnt, want[2])
    # within every column the 1-saddles ascend
    seg = np.repeat(np.arange(n2), np.diff(colptr))
    assert np.all((np.diff(row.astype(np.int64)) > 0) | (np.diff(seg) > 0))


def test_csc_after_field_change():
    """The column form follows the plan's latest pass."""
    m = msc()
    a = fields.grf((30, 30, 30), 3.0, seed=41)
    b = fields.grf((30, 30, 30), 3.0, seed=42)
    plan = m.Plan(dims_of(a))
    for f in (a, b, a):
        m.msc_compute(plan, gpu_field(f))
        counts, _ = m.msc_critical(plan)
        rowptr, col, cnt = (to_np(x) for x in m.msc_saddle_arcs(plan))
        colptr, row, ccnt = (to_np(x) for x in m.msc_saddle_arcs_csc(plan))
        want = _transpose(int(counts[2]), rowptr, col, cnt)
        assert np.array_equal(colptr, want[0]) and np.array_equal(row, want[1]) and np.array_equal(ccnt, want[2])
