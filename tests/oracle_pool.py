"""Whole-volume oracle runs for a process pool (test infrastructure).  Kept free of torch and of
the CUDA library so that spawned workers import only the oracle and numpy."""
from __future__ import annotations

import numpy as np

import oracle


def critical_counts(f: np.ndarray) -> list:
    """Critical cells per dimension of the oracle's lower-star gradient of f."""
    nz, ny, nx = f.shape
    pair = oracle.gradient(f)
    counts, _ = oracle.critical((nx, ny, nz), pair)
    return [int(c) for c in counts]
