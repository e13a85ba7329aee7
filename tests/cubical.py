"""Plain-Python cubical complex of a small 3D grid, for the oracle's pins.

Independent of both the oracle (C++) and the CUDA library: cells are written out by
coordinates on the refined grid (2nx-1)x(2ny-1)x(2nz-1) as in Sec. 2.2 of the paper
(a cell of dimension i has i odd coordinates; facets change one odd coordinate by 1).
"""
from __future__ import annotations

import itertools

import numpy as np


class Complex:
    def __init__(self, dims):
        self.nx, self.ny, self.nz = (int(v) for v in dims)
        self.r = (2 * self.nx - 1, 2 * self.ny - 1, 2 * self.nz - 1)

    # --- ids -----------------------------------------------------------------------
    def cid(self, c):
        rx, ry, _ = self.r
        return c[0] + rx * (c[1] + ry * c[2])

    def coords(self, i):
        rx, ry, _ = self.r
        return (i % rx, (i // rx) % ry, i // (rx * ry))

    def ncells(self):
        return self.r[0] * self.r[1] * self.r[2]

    def cells(self):
        return range(self.ncells())

    def inside(self, c):
        return all(0 <= c[k] < self.r[k] for k in range(3))

    def dim(self, i):
        return sum(v & 1 for v in self.coords(i))

    def vid(self, x, y, z):
        return x + self.nx * (y + self.ny * z)

    # --- incidence -------------------------------------------------------------------
    def vertices(self, i):
        c = self.coords(i)
        axes = [((v - 1) // 2, (v + 1) // 2) if v & 1 else (v // 2,) for v in c]
        return [self.vid(x, y, z) for z in axes[2] for y in axes[1] for x in axes[0]]

    def facets(self, i):
        c = self.coords(i)
        out = []
        for k in range(3):
            if c[k] & 1:
                for s in (-1, 1):
                    d = list(c)
                    d[k] += s
                    out.append(self.cid(d))
        return out

    def cofacets(self, i):
        c = self.coords(i)
        out = []
        for k in range(3):
            if not c[k] & 1:
                for s in (-1, 1):
                    d = list(c)
                    d[k] += s
                    if self.inside(d):
                        out.append(self.cid(d))
        return out


def vertex_rank(f: np.ndarray) -> np.ndarray:
    """Rank of each vertex in the order (value, index); f is [nz, ny, nx]."""
    flat = f.reshape(-1).astype(np.float64)
    order = np.lexsort((np.arange(flat.size), flat))
    rank = np.empty(flat.size, dtype=np.int64)
    rank[order] = np.arange(flat.size)
    return rank


def pairs_dict(pair: np.ndarray) -> dict:
    """{cell: partner} for paired cells of an oracle pairing array (0xFFFFFFFF = critical)."""
    idx = np.nonzero(pair != 0xFFFFFFFF)[0]
    return {int(i): int(pair[i]) for i in idx}


def random_field(shape_zyx, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal(shape_zyx).astype(np.float32)
    if kind == "ties":  # few distinct values: exercises the index tie-break
        return rng.integers(0, 3, size=shape_zyx).astype(np.float32)
    if kind == "near":  # 1 + k ulp, k < 64: order keys that differ only in their lowest bits, and ties
        ulp = np.float32(2.0 ** -23)
        return (np.float32(1.0) + rng.integers(0, 64, size=shape_zyx).astype(np.float32) * ulp).astype(np.float32)
    raise KeyError(kind)


def product_shapes(max_n=4):
    return [s for s in itertools.product(range(2, max_n + 1), repeat=3)]
