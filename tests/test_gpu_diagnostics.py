"""Per-stage diagnostics (the statistics of Sec. 4.2 "performance analysis": critical points,
saddles, junction nodes, sparsity ratios of A, B, B*, D and D*, product-loop iterations) as the
library reports them after a run, against the same quantities counted from the oracle's outputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc

pytestmark = pytest.mark.gpu

CASES = [("cos32", fields.cosine_lattice()), ("grf40", fields.grf((40, 40, 40), 3.0, seed=12)),
         ("grf24x40x33", fields.grf((24, 40, 33), 2.5, seed=7)),
         ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5)),
         ("normal9x8x33", random_field((9, 8, 33), 905, "normal")), ("ties6", random_field((6, 6, 6), 952, "ties"))]


def _oracle_stats(f):
    e = oracle.compute_all(f, with_minor=True, with_dstar=True)
    mn = e["minor"]
    dstar = e["dstar"]
    return dict(counts=[int(c) for c in e["counts"]],
                n_reachable=int(sum(bin(int(v)).count("1") for v in e["visited"].reshape(-1))),
                n_bfs_levels=int(e["levels"]), n_junctions=len(e["junctions"]),
                nnz_A=len(mn["A"][0]), nnz_B=len(mn["B"][0]), nnz_Bstar=len(mn["Bstar"][0]), nnz_D=len(mn["D"][0]),
                nnz_Dstar=len(dstar[0]), n_iter=int(e["n_iter"]),
                max_path_count=int(dstar[2].max()) if len(dstar[2]) else 0)


@pytest.mark.parametrize("name,f", CASES, ids=[n for n, _ in CASES])
@pytest.mark.parametrize("method", [1, 2])
def test_stats_match_oracle(name, f, method):
    m = msc()
    plan = m.Plan(dims_of(f), path_count_method=method)
    m.msc_compute(plan, gpu_field(f))
    got = m.msc_get_stats(plan)
    want = _oracle_stats(f)
    for k, v in want.items():
        assert (list(got[k]) if k == "counts" else int(got[k])) == v, k
    dg, dw = m.diagnostics(got), m.diagnostics(dict(want, peak_device_bytes=got["peak_device_bytes"]))
    assert dg == dw
    # Sec. 4.2's observations, as invariants: D* holds D, so it is no sparser
    if dg["sparsity"]["D"] is not None:
        assert dg["sparsity"]["Dstar"] <= dg["sparsity"]["D"]
