"""Parity of stages (a1) lower-star gradient and (a2) critical cells: CUDA path (through the
C ABI) vs the CPU oracle, bit-exact."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from synth import fields
from tests.cubical import random_field
from tests.gpu_util import dims_of, msc, run_gradient

pytestmark = pytest.mark.gpu


def _small_fields():
    out = [("cos32", fields.cosine_lattice())]
    shapes = [(2, 2, 2), (3, 5, 7), (9, 8, 33), (10, 9, 34), (17, 16, 65), (20, 40, 70), (5, 3, 100), (64, 1 + 1, 3)]
    for i, shp in enumerate(shapes):
        out.append((f"normal{shp}", random_field(shp, 700 + i, "normal")))
        out.append((f"ties{shp}", random_field(shp, 800 + i, "ties")))
    out.append(("grf48", fields.grf((48, 48, 48), 3.0, seed=11)))
    out.append(("blobs40", fields.gaussian_blobs(n=40, n_blobs=12, sigma_range=(2, 6), seed=4)))
    inf = random_field((6, 7, 8), 3)
    inf[0, 0, 0], inf[5, 6, 7], inf[2, 3, 4] = -np.inf, np.inf, np.inf
    inf[1, 1, 1] = -0.0
    inf[1, 1, 2] = 0.0
    out.append(("inf_zero", inf))
    return out


@pytest.mark.parametrize("name,f", _small_fields(), ids=[n for n, _ in _small_fields()])
def test_gradient_and_critical_match_oracle(name, f):
    d = dims_of(f)
    pair = oracle.gradient(f)
    want_words = oracle.pack(d, pair)
    want_counts, want_lists = oracle.critical(d, pair)
    _, words, counts, lists, _ = run_gradient(f)
    assert np.array_equal(words, want_words), f"{int((words != want_words).sum())} packed words differ"
    assert counts == [int(c) for c in want_counts]
    for k in range(4):
        assert np.array_equal(lists[k], want_lists[k]), f"critical {k}-cells differ"


def test_plan_reuse_and_repeat():
    f1 = random_field((12, 13, 40), 1)
    f2 = random_field((12, 13, 40), 2)
    m = msc()
    plan = m.Plan(dims_of(f1))
    for f in (f1, f2, f1):
        _, words, counts, lists, _ = run_gradient(f, plan)
        pair = oracle.gradient(f)
        assert np.array_equal(words, oracle.pack(dims_of(f), pair))
        assert counts == [int(c) for c in oracle.critical(dims_of(f), pair)[0]]


def test_nan_is_rejected():
    f = random_field((8, 8, 8), 5)
    f[3, 4, 5] = np.nan
    m = msc()
    with pytest.raises(m.MscError) as e:
        run_gradient(f)
    assert e.value.status == 2


def test_bad_arguments():
    m = msc()
    with pytest.raises(m.MscError):
        m.Plan((1, 4, 4))
    plan = m.Plan((4, 4, 4))
    with pytest.raises(m.MscError) as e:
        m.msc_critical(plan)  # before msc_gradient
    assert e.value.status == 11


TILES = [(8, 8, 512), (8, 4, 256), (4, 8, 256), (8, 16, 512), (16, 8, 512), (16, 8, 1024), (16, 16, 512),
         (8, 8, 256), (16, 8, 256)]


@pytest.mark.parametrize("tile", range(1, len(TILES) + 1))
def test_every_tile_variant_matches_oracle(tile):
    """The autotuner chooses among tile variants; each must compute the same words (ragged tiles
    on every axis, ties, a smooth field)."""
    m = msc()
    cases = [random_field((17, 9, 35), 40 + tile, "normal"), random_field((9, 18, 33), 50 + tile, "ties"),
             random_field((11, 20, 37), 60 + tile, "near"), fields.grf((24, 21, 70), 3.0, seed=tile)]
    for f in cases:
        plan = m.Plan(dims_of(f), gradient_tile=tile)
        _, words, counts, lists, _ = run_gradient(f, plan)
        pair = oracle.gradient(f)
        assert np.array_equal(words, oracle.pack(dims_of(f), pair))
        assert counts == [int(c) for c in oracle.critical(dims_of(f), pair)[0]]
        st = m.msc_get_stats(plan)["gradient_tile"]
        assert (st & 0xFF, (st >> 8) & 0xFF, st >> 16) == TILES[tile - 1]


@pytest.mark.parametrize("tile", range(1, len(TILES) + 1))
def test_words_are_rewritten_whatever_the_buffer_held(tile):
    """Only the tiles' face words (the ones finished with atomicOr) are zeroed before the lower-star
    kernel; every other word must get a plain store.  Fill the plan's word buffer with all-ones
    first (a buffer from an earlier field holds arbitrary codes) and check every word afterwards,
    on grids that end inside a tile on every axis and on grids that end on a tile boundary."""
    m = msc()
    for shp in ((19, 21, 45), (16, 16, 64), (33, 17, 95)):
        f = random_field(shp, 90 + tile)
        plan = m.Plan(dims_of(f), gradient_tile=tile)
        run_gradient(f, plan)
        m.msc_gradient_words(plan).view(torch.int32).fill_(-1)
        _, words, counts, _, _ = run_gradient(f, plan)
        pair = oracle.gradient(f)
        assert np.array_equal(words, oracle.pack(dims_of(f), pair)), shp
        assert counts == [int(c) for c in oracle.critical(dims_of(f), pair)[0]]


def test_tile_option_is_validated():
    m = msc()
    with pytest.raises(m.MscError):
        m.Plan((8, 8, 8), gradient_tile=len(TILES) + 1)
