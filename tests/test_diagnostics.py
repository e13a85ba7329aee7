"""The diagnostics helper (host arithmetic only): sparsity ratio = zero entries / all entries of
each matrix of the minor and of D*, with the matrix shapes fixed by the critical and junction
counts (Sec. 4.2 "Matrix sparsity")."""
from __future__ import annotations

import pytest


def _m():
    from paper_2009_03707_gb300 import msc
    return msc


def _stats(**kw):
    s = dict(counts=[1, 2, 3, 1], n_junctions=4, nnz_A=2, nnz_B=1, nnz_Bstar=6, nnz_D=3, nnz_Dstar=6, n_iter=3,
             max_path_count=5, n_bfs_levels=4, peak_device_bytes=100)
    s.update(kw)
    return s


def test_shapes_and_ratios():
    pytest.importorskip("torch")
    d = _m().diagnostics(_stats())
    assert d["critical"] == 7 and d["saddles"] == 5 and d["extrema"] == 2 and d["junctions"] == 4
    assert d["junctions_per_critical"] == pytest.approx(4 / 7)
    sp = d["sparsity"]
    # A: 2 x 4, B: 4 x 4, B*: 4 x 3, D and D*: 2 x 3
    assert sp["A"] == pytest.approx(6 / 8) and sp["B"] == pytest.approx(15 / 16)
    assert sp["Bstar"] == pytest.approx(6 / 12) and sp["D"] == pytest.approx(3 / 6) and sp["Dstar"] == 0.0
    assert d["n_iter"] == 3 and d["max_path_count"] == 5


def test_empty_shapes():
    pytest.importorskip("torch")
    d = _m().diagnostics(_stats(counts=[1, 0, 0, 0], n_junctions=0, nnz_A=0, nnz_B=0, nnz_Bstar=0, nnz_D=0,
                                nnz_Dstar=0, n_iter=0, max_path_count=0))
    assert all(v is None for v in d["sparsity"].values()) and d["junctions_per_critical"] == 0.0
