"""Parity of stages (a3)-(a6) through the C ABI against the CPU oracle, bit-exact:
extremum labels and arcs, reachability (visited bitmap and level count), junctions, the
minor matrices A, B, B*, D, and the saddle-saddle path counts D*."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import csr_to_coo, dims_of, edge_layout, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _cases():
    out = [("cos32", fields.cosine_lattice()), ("grf40", fields.grf((40, 40, 40), 3.0, seed=12)),
           ("grf25x30x70", fields.grf((25, 30, 70), 2.5, seed=13)),
           ("blobs36", fields.gaussian_blobs(n=36, n_blobs=10, sigma_range=(2, 6), seed=5))]
    for i, shp in enumerate([(2, 2, 2), (3, 4, 5), (6, 6, 6), (9, 8, 33), (5, 3, 65)]):
        out.append((f"normal{shp}", random_field(shp, 900 + i, "normal")))
        out.append((f"ties{shp}", random_field(shp, 950 + i, "ties")))
    return out


CASES = _cases()


@pytest.fixture(scope="module")
def results():
    m = msc()
    res = {}
    for name, f in CASES:
        plan = m.Plan(dims_of(f))
        d = gpu_field(f)
        m.msc_compute(plan, d)
        counts, cells = m.msc_critical(plan)
        amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
        vis, levels = m.msc_reachability(plan)
        junc = m.msc_junctions(plan)
        minor = [tuple(to_np(x) for x in m.msc_minor(plan, w)) for w in range(4)]
        dstar = tuple(to_np(x) for x in m.msc_saddle_arcs(plan))
        res[name] = dict(counts=counts, cells=[to_np(c) for c in cells], min_arcs=to_np(amin),
                         max_arcs=to_np(amax), vmin=to_np(vmin), cmax=to_np(cmax), visited=to_np(vis),
                         levels=levels, junctions=to_np(junc), minor=minor, dstar=dstar,
                         stats=m.msc_get_stats(plan))
    return res


@pytest.fixture(scope="module")
def expected():
    return {name: oracle.compute_all(f) for name, f in CASES}


IDS = [n for n, _ in CASES]


@pytest.mark.parametrize("name", IDS)
def test_extremum(name, results, expected):
    r, e = results[name], expected[name]
    assert np.array_equal(r["vmin"], e["vertex_min"])
    assert np.array_equal(r["cmax"], e["cube_max"])
    assert np.array_equal(r["min_arcs"], e["min_arcs"])
    assert np.array_equal(r["max_arcs"], e["max_arcs"])


@pytest.mark.parametrize("name", IDS)
def test_reachability(name, results, expected):
    r, e = results[name], expected[name]
    assert np.array_equal(r["visited"], edge_layout(e["visited"]))
    assert r["levels"] == e["levels"]
    assert r["stats"]["n_reachable"] == int(sum(bin(int(v)).count("1") for v in e["visited"].reshape(-1)))


@pytest.mark.parametrize("name", IDS)
def test_junctions_and_minor(name, results, expected):
    r, e = results[name], expected[name]
    assert np.array_equal(r["junctions"], e["junctions"])
    for w, key in enumerate(oracle.MINOR_NAMES):
        rows, cols, mult = csr_to_coo(*r["minor"][w])
        er, ec, em = e["minor"][key]
        assert np.array_equal(rows, er) and np.array_equal(cols, ec), key
        assert np.array_equal(mult.astype(np.uint64), em), key


@pytest.mark.parametrize("name", IDS)
def test_dstar(name, results, expected):
    r, e = results[name], expected[name]
    rows, cols, cnt = csr_to_coo(*r["dstar"])
    er, ec, en = e["dstar"]
    assert np.array_equal(rows, er)
    assert np.array_equal(cols, ec)
    assert np.array_equal(cnt, en)
    assert r["stats"]["n_iter"] == e["n_iter"]
    assert r["stats"]["nnz_Dstar"] == len(er)


@pytest.mark.parametrize("tier", [0, 1, 2])
@pytest.mark.parametrize("name", ["grf40", "grf25x30x70", "cos32", "ties(9, 8, 33)", "blobs36"])
def test_dstar_row_wise_every_tier(name, tier, expected):
    """The paper's iteration A <- A B, run row by row from each tier (register, warp-table and
    CTA-table), gives the same D* and iteration count as the junction waves and the oracle."""
    m = msc()
    f = dict(CASES)[name]
    plan = m.Plan(dims_of(f), path_count_tier=tier, path_count_method=1)
    m.msc_compute(plan, gpu_field(f))
    rows, cols, cnt = csr_to_coo(*(to_np(x) for x in m.msc_saddle_arcs(plan)))
    er, ec, en = expected[name]["dstar"]
    assert np.array_equal(rows, er) and np.array_equal(cols, ec) and np.array_equal(cnt, en)
    assert m.msc_get_stats(plan)["n_iter"] == expected[name]["n_iter"]


def test_dstar_methods_agree_on_long_path_networks():
    """A blob field with long V-path networks (many junction levels, large multiplicities):
    junction waves, row-wise products and the oracle agree entry by entry."""
    m = msc()
    f = fields.gaussian_blobs(n=44, n_blobs=6, sigma_range=(4, 12), seed=9)
    e = oracle.compute_all(f, with_minor=True, with_dstar=True)
    got = {}
    for method in (1, 2):
        plan = m.Plan(dims_of(f), path_count_method=method)
        m.msc_compute(plan, gpu_field(f))
        got[method] = csr_to_coo(*(to_np(x) for x in m.msc_saddle_arcs(plan)))
        assert m.msc_get_stats(plan)["n_iter"] == e["n_iter"]
    er, ec, en = e["dstar"]
    for method in (1, 2):
        rows, cols, cnt = got[method]
        assert np.array_equal(rows, er) and np.array_equal(cols, ec) and np.array_equal(cnt, en)


def test_dstar_row_wise_counts_beyond_one_byte():
    """Tier 0 keeps a count in 8 bits beside its key when the ranks fit in 24; a row whose counts
    pass 255 must go on to the 32-bit tiers.  This blob field has rows with counts in the
    thousands, and the row-wise products must still give the oracle's D*."""
    m = msc()
    f = fields.gaussian_blobs(n=48, n_blobs=3, sigma_range=(10, 20), seed=2)
    e = oracle.compute_all(f, with_minor=False, with_dstar=True)
    er, ec, en = e["dstar"]
    assert en.max() > 255
    plan = m.Plan(dims_of(f), path_count_tier=0, path_count_method=1)
    for _ in range(3):  # synchronised, then replayed
        m.msc_compute(plan, gpu_field(f))
        rows, cols, cnt = csr_to_coo(*(to_np(x) for x in m.msc_saddle_arcs(plan)))
        assert np.array_equal(rows, er) and np.array_equal(cols, ec) and np.array_equal(cnt, en)
        assert m.msc_get_stats(plan)["max_path_count"] == int(en.max())
