"""Host-side pieces of bench.py that need no GPU: the CPU baseline's sampling of the oracle."""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    return bench


def test_cpu_baseline_samples_whole_small_fields_and_blocks_of_large_ones():
    bench = _bench()
    rng = np.random.default_rng(3)
    small = rng.standard_normal((12, 10, 9)).astype(np.float32)
    line = bench.cpu_baseline(small, min_seconds=0.0)
    assert line["kind"] == "oracle" and line["cores"] == 1 and line["unit"] == "Mvoxel/s"
    assert line["value"] > 0 and "the whole field" in line["sample"] and "1 oracle run" in line["sample"]
    # a field taller than one 64-plane block: successive blocks until the time bound, cycling
    tall = rng.standard_normal((70, 8, 8)).astype(np.float32)
    line = bench.cpu_baseline(tall, min_seconds=1e9, max_runs=3)
    assert "blocks of at most 64x96x96" in line["sample"] and "3 oracle run(s)" in line["sample"]
    assert f"over {64 * 64 + 6 * 64 + 64 * 64} voxels" in line["sample"]
