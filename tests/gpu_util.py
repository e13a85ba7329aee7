"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding and bring
results back as numpy arrays for element-by-element comparison with the oracle."""
from __future__ import annotations

import numpy as np
import torch

NONE = 0xFFFFFFFF


def msc():
    from paper_2009_03707_gb300 import msc as m
    return m


def to_np(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


def dims_of(f: np.ndarray):
    nz, ny, nx = f.shape
    return (nx, ny, nz)


def gpu_field(f: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()


def run_gradient(f: np.ndarray, plan=None):
    m = msc()
    plan = plan or m.Plan(dims_of(f))
    d = gpu_field(f)
    m.msc_gradient(plan, d)
    counts, cells = m.msc_critical(plan)
    words = to_np(m.msc_gradient_words(plan))
    return plan, words, counts, [to_np(c) for c in cells], d


def edge_layout(visited_per_vertex: np.ndarray) -> np.ndarray:
    """Oracle visited flags (bit a of [z,y,x] = 1-cell along axis a) -> the library's 1-cell
    row bitmap: word (((z*2 + c)*ny + y)*2 + b)*W + (x >> 5), bit x & 31, with (b, c) =
    (0,0) for x-edges, (1,0) for y-edges, (0,1) for z-edges."""
    nz, ny, nx = visited_per_vertex.shape
    W = (nx + 31) // 32
    out = np.zeros((nz, 2, ny, 2, W), dtype=np.uint64)
    xs = np.arange(nx)
    for axis, (b, c) in enumerate(((0, 0), (1, 0), (0, 1))):
        bits = ((visited_per_vertex >> axis) & 1).astype(np.uint64)  # [z, y, x]
        vals = bits << (xs & 31).astype(np.uint64)[None, None, :]
        for w in range(W):
            out[:, c, :, b, w] = vals[:, :, w * 32:(w + 1) * 32].sum(axis=2)
    return out.reshape(-1).astype(np.uint32)


def csr_to_coo(rowptr: np.ndarray, col: np.ndarray, val: np.ndarray):
    rows = np.repeat(np.arange(len(rowptr) - 1, dtype=np.uint32), np.diff(rowptr.astype(np.int64)))
    return rows, col, val
