"""Simplification of the 1-skeleton (Sec. 4) on the GPU, in rounds of independent cancellations:
msc_simplify against the oracle's restatement of the same rounds, element by element (survivors,
the cancellation log round by round, the remaining arcs with their multiplicities), and against
the oracle's serial persistence order, which ends in the same complex on these fields."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def _two_wells():
    x = np.arange(31)[None, None, :]
    y = np.arange(9)[None, :, None]
    z = np.arange(9)[:, None, None]
    return (np.minimum((x - 8.0) ** 2, (x - 22.0) ** 2 + 10.0) + (y - 4.0) ** 2 + (z - 4.0) ** 2).astype(np.float32)


def _cases():
    out = [("cos32", fields.cosine_lattice()), ("wells", _two_wells()),
           ("grf28", fields.grf((28, 26, 30), 3.0, seed=14)),
           ("blobs30", fields.gaussian_blobs(n=30, n_blobs=9, sigma_range=(2, 5), seed=6))]
    for i, shp in enumerate([(4, 5, 6), (3, 7, 9), (9, 8, 20)]):
        out.append((f"normal{shp}", random_field(shp, 1000 + i, "normal")))
        out.append((f"ties{shp}", random_field(shp, 1050 + i, "ties")))
    return out


def _gpu(f, thresholds):
    m = msc()
    plan = m.Plan(dims_of(f))
    d = gpu_field(f)
    m.msc_compute(plan, d)
    out = []
    for th in thresholds:
        r = m.msc_simplify(plan, d, th)
        nodeptr, adj, mult = to_np(r["nodeptr"]), to_np(r["adj"]), to_np(r["mult"])
        u = np.repeat(np.arange(len(nodeptr) - 1), np.diff(nodeptr))
        keep = u < adj
        out.append(dict(r, alive=to_np(r["alive"]).astype(bool), log=to_np(r["log"]),
                        arcs=sorted(zip(u[keep].tolist(), adj[keep].tolist(), mult[keep].tolist())),
                        sym=np.array_equal(np.sort(u * (len(nodeptr)) + adj), np.sort(adj.astype(np.int64) * len(nodeptr) + u))))
    return out


@pytest.mark.parametrize("name,f", _cases(), ids=[n for n, _ in _cases()])
def test_simplification_matches_oracle_rounds(name, f):
    sk = oracle.skeleton(f)
    pers = np.abs(sk["value"][sk["arc_u"]] - sk["value"][sk["arc_v"]])
    ths = [0.0, float(np.percentile(pers, 25)) if len(pers) else 0.0, float(np.median(pers)) if len(pers) else 0.0, 1e9]
    for th, g in zip(ths, _gpu(f, ths)):
        want = oracle.simplify(sk, th, rounds=True)
        assert g["n_rounds"] == want["n_rounds"]
        assert np.array_equal(g["alive"], want["alive"])
        assert np.array_equal(g["log"][:, 0], want["upper"]) and np.array_equal(g["log"][:, 1], want["lower"])
        assert np.array_equal(g["log"][:, 2], want["round"])
        assert g["arcs"] == sorted(zip(want["arc_u"].tolist(), want["arc_v"].tolist(), want["arc_mult"].tolist()))
        assert g["sym"]
        assert g["counts"] == [int(c) for c in np.bincount(sk["index"][want["alive"]], minlength=4)]
        serial = oracle.simplify(sk, th)
        assert np.array_equal(serial["alive"], want["alive"])


@pytest.mark.slow
def test_anisotropic_batch_volume():
    """The smallest volume of the uneven batch (seed 126, 91 x 48 x 61): rounds against the oracle at the
    median persistence, and the serial order's survivors."""
    f = fields.batch_volume(126)
    sk = oracle.skeleton(f)
    th = float(np.median(np.abs(sk["value"][sk["arc_u"]] - sk["value"][sk["arc_v"]])))
    (g,) = _gpu(f, [th])
    want = oracle.simplify(sk, th, rounds=True)
    assert g["n_rounds"] == want["n_rounds"] and np.array_equal(g["alive"], want["alive"])
    assert np.array_equal(g["log"][:, 0], want["upper"]) and np.array_equal(g["log"][:, 1], want["lower"])
    assert g["arcs"] == sorted(zip(want["arc_u"].tolist(), want["arc_v"].tolist(), want["arc_mult"].tolist()))
    assert np.array_equal(oracle.simplify(sk, th)["alive"], want["alive"])


def test_closed_forms():
    (g,) = _gpu(_two_wells(), [39.0])
    assert g["counts"] == [1, 0, 0, 0] and g["n_cancelled"] == 1
    lo, hi = _gpu(fields.cosine_lattice(), [1.99, 2.01])
    assert lo["counts"] == [8, 12, 6, 1] and lo["n_cancelled"] == 0
    assert hi["counts"] == [1, 0, 0, 0] and hi["n_cancelled"] == 13


@pytest.mark.slow
def test_grf64_against_oracle_and_grf256_invariants():
    f = fields.grf((64, 64, 64), 3.0, seed=15)
    sk = oracle.skeleton(f)
    (g,) = _gpu(f, [0.2])
    want = oracle.simplify(sk, 0.2, rounds=True)
    assert np.array_equal(g["alive"], want["alive"]) and g["n_rounds"] == want["n_rounds"]
    assert g["arcs"] == sorted(zip(want["arc_u"].tolist(), want["arc_v"].tolist(), want["arc_mult"].tolist()))
    # the bench workload after replayed passes: the Euler characteristic of a box stays 1, every
    # cancellation removes one point of each of two consecutive indices, and counts only fall
    m = msc()
    f = fields.config_field("grf256")
    plan = m.Plan(dims_of(f))
    d = gpu_field(f)
    for _ in range(3):
        m.msc_compute(plan, d)
    counts, _ = m.msc_critical(plan)
    for th in (0.05, 0.5):
        r = m.msc_simplify(plan, d, th)
        c = r["counts"]
        assert c[0] - c[1] + c[2] - c[3] == 1
        assert all(a <= b for a, b in zip(c, counts)) and sum(counts) - sum(c) == 2 * r["n_cancelled"]
        log = to_np(r["log"])
        idx = np.searchsorted(np.cumsum(counts), log[:, :2], side="right")
        assert np.all(idx[:, 0] == idx[:, 1] + 1)
