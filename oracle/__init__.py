"""TEST INFRASTRUCTURE ONLY: ctypes wrapper around the plain CPU oracle (msc_oracle.cpp).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline legs may import
this package. It shares no code with the CUDA library and never loads it.

Arrays follow the library's conventions: a field is float32 [nz, ny, nx]; dims are
(nx, ny, nz); cells are ids on the refined grid (2nx-1)x(2ny-1)x(2nz-1).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msc_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmsc_oracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF
STATUS = {0: "ok", 1: "bad argument", 2: "NaN in field", 4: "grid too large for 32-bit cell ids",
          6: "path count overflows uint64", 9: "internal error"}


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what}: status {status} ({STATUS.get(status, '?')})")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_SIGNATURES = {
    "ora_version": ([], ctypes.c_int),
    "ora_gradient": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "ora_packed_at": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ora_pack": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "ora_critical_counts": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "ora_critical_list": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "ora_extremum_labels": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "ora_min_arcs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ora_max_arcs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ora_reachable": ([ctypes.c_void_p] * 3, ctypes.c_int64),
    "ora_junctions": ([ctypes.c_void_p] * 4, ctypes.c_int64),
    "ora_minor": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_int64, ctypes.c_void_p], ctypes.c_void_p),
    "ora_minor_status": ([ctypes.c_void_p], ctypes.c_int),
    "ora_minor_size": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int64),
    "ora_minor_copy": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], None),
    "ora_minor_free": ([ctypes.c_void_p], None),
    "ora_path_counts": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_void_p),
    "ora_result_status": ([ctypes.c_void_p], ctypes.c_int),
    "ora_result_size": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_result_copy": ([ctypes.c_void_p] * 4, None),
    "ora_result_free": ([ctypes.c_void_p], None),
    "ora_n_iter": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p],
                   ctypes.c_int64),
    "ora_lazy_pairs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ora_lazy_vertex_min": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p],
                            ctypes.c_int),
    "ora_lazy_cube_max": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p],
                          ctypes.c_int),
    "ora_lazy_nodes": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ora_lazy_dstar_rows": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_void_p),
    "ora_arc_cells": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_void_p], ctypes.c_void_p),
    "ora_ss_arc_cells": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_void_p),
    "ora_arc_status": ([ctypes.c_void_p], ctypes.c_int),
    "ora_arc_count": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_arc_cells_size": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_arc_copy": ([ctypes.c_void_p] * 3, None),
    "ora_arc_free": ([ctypes.c_void_p], None),
    "ora_simplify": ([ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double], ctypes.c_void_p),
    "ora_simplify_status": ([ctypes.c_void_p], ctypes.c_int),
    "ora_simplify_cancelled": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_simplify_arcs": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_simplify_copy": ([ctypes.c_void_p] * 8, None),
    "ora_simplify_free": ([ctypes.c_void_p], None),
    "ora_simplify_rounds": ([ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double], ctypes.c_void_p),
    "ora_simplify_rounds_count": ([ctypes.c_void_p], ctypes.c_int64),
    "ora_simplify_rounds_of": ([ctypes.c_void_p, ctypes.c_void_p], None),
}


def _bind(path: str):
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


@contextlib.contextmanager
def swap_library(path: str):
    """Run the wrappers against another build of the oracle (used to test that pins fail on
    deliberately broken copies of the source)."""
    global _lib
    old = _load()
    _lib = _bind(path)
    try:
        yield
    finally:
        _lib = old


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(f_or_dims):
    if isinstance(f_or_dims, np.ndarray) and f_or_dims.ndim == 3:
        nz, ny, nx = f_or_dims.shape
        return np.array([nx, ny, nz], dtype=np.int64)
    return np.asarray(f_or_dims, dtype=np.int64).reshape(3)


def refined_shape(dims):
    nx, ny, nz = (int(v) for v in dims)
    return (2 * nz - 1, 2 * ny - 1, 2 * nx - 1)


def gradient(f: np.ndarray) -> np.ndarray:
    """Partner cell id per cell (0xFFFFFFFF = critical), flat over the refined grid."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    d = _dims(f)
    n = int(np.prod(refined_shape(d)))
    pair = np.empty(n, dtype=np.uint32)
    st = _load().ora_gradient(_p(d), _p(f), _p(pair))
    if st:
        raise OracleError(st, "gradient")
    return pair


def packed_at(f: np.ndarray, verts) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float32)
    d = _dims(f)
    verts = np.ascontiguousarray(verts, dtype=np.int64)
    out = np.empty(len(verts), dtype=np.uint32)
    st = _load().ora_packed_at(_p(d), _p(f), len(verts), _p(verts), _p(out))
    if st:
        raise OracleError(st, "packed_at")
    return out


def pack(dims, pair) -> np.ndarray:
    d = _dims(dims)
    nx, ny, nz = (int(v) for v in d)
    out = np.empty((nz, ny, nx), dtype=np.uint32)
    st = _load().ora_pack(_p(d), _p(pair), _p(out))
    if st:
        raise OracleError(st, "pack")
    return out


def critical(dims, pair):
    d = _dims(dims)
    lib = _load()
    counts = np.zeros(4, dtype=np.int64)
    lib.ora_critical_counts(_p(d), _p(pair), _p(counts))
    lists = []
    for k in range(4):
        out = np.empty(int(counts[k]), dtype=np.uint32)
        if counts[k]:
            lib.ora_critical_list(_p(d), _p(pair), k, _p(out))
        lists.append(out)
    return counts, lists


def extremum(dims, pair, s1, s2):
    d = _dims(dims)
    nx, ny, nz = (int(v) for v in d)
    lib = _load()
    vmin = np.empty((nz, ny, nx), dtype=np.uint32)
    cmax = np.empty((nz, ny, nx), dtype=np.uint32)
    st = lib.ora_extremum_labels(_p(d), _p(pair), _p(vmin), _p(cmax))
    if st:
        raise OracleError(st, "extremum_labels")
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    s2 = np.ascontiguousarray(s2, dtype=np.uint32)
    amin = np.empty(2 * len(s1), dtype=np.uint32)
    amax = np.empty(2 * len(s2), dtype=np.uint32)
    lib.ora_min_arcs(_p(d), _p(vmin), len(s1), _p(s1), _p(amin))
    lib.ora_max_arcs(_p(d), _p(cmax), len(s2), _p(s2), _p(amax))
    return vmin, cmax, amin, amax


def arc_cells(dims, pair, s1, s2):
    """The cells along every saddle-extremum arc (Sec. 3.4): (offsets int64[n_arcs + 1], cells
    uint32), arcs ordered as the arc lists (2 per 1-saddle, then 2 per 2-saddle)."""
    d = _dims(dims)
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    s2 = np.ascontiguousarray(s2, dtype=np.uint32)
    lib = _load()
    h = lib.ora_arc_cells(_p(d), _p(pair), len(s1), _p(s1), len(s2), _p(s2))
    try:
        st = lib.ora_arc_status(h)
        if st:
            raise OracleError(st, "arc_cells")
        offsets = np.empty(lib.ora_arc_count(h) + 1, dtype=np.int64)
        cells = np.empty(lib.ora_arc_cells_size(h), dtype=np.uint32)
        lib.ora_arc_copy(h, _p(offsets), _p(cells))
    finally:
        lib.ora_arc_free(h)
    return offsets, cells


def ss_arc_cells(dims, pair, s1, s2, dstar):
    """The cells along every saddle-saddle arc of multiplicity 1 (Sec. 3.3): for each D* entry
    (dstar = (rows, cols, counts), sorted by row then column) the V-path from its 1-saddle to its
    2-saddle -- s, then (quad, 1-cell) per step, then t -- or nothing when the count is not 1.
    Returns (offsets int64[nnz + 1], cells uint32)."""
    d = _dims(dims)
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    s2 = np.ascontiguousarray(s2, dtype=np.uint32)
    rows, cols, cnt = dstar
    rows = np.asarray(rows, dtype=np.int64)
    rowptr = np.ascontiguousarray(np.searchsorted(rows, np.arange(len(s1) + 1)), dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    cnt = np.ascontiguousarray(cnt, dtype=np.uint64)
    lib = _load()
    h = lib.ora_ss_arc_cells(_p(d), _p(pair), len(s1), _p(s1), len(s2), _p(s2), _p(rowptr), _p(cols), _p(cnt))
    try:
        st = lib.ora_arc_status(h)
        if st:
            raise OracleError(st, "ss_arc_cells")
        offsets = np.empty(lib.ora_arc_count(h) + 1, dtype=np.int64)
        cells = np.empty(lib.ora_arc_cells_size(h), dtype=np.uint32)
        lib.ora_arc_copy(h, _p(offsets), _p(cells))
    finally:
        lib.ora_arc_free(h)
    return offsets, cells


def reachable(dims, pair):
    d = _dims(dims)
    nx, ny, nz = (int(v) for v in d)
    vis = np.empty((nz, ny, nx), dtype=np.uint8)
    levels = _load().ora_reachable(_p(d), _p(pair), _p(vis))
    if levels < 0:
        raise OracleError(int(-levels), "reachable")
    return vis, int(levels)


def junctions(dims, pair, visited):
    d = _dims(dims)
    lib = _load()
    n = lib.ora_junctions(_p(d), _p(pair), _p(visited), None)
    out = np.empty(n, dtype=np.uint32)
    if n:
        lib.ora_junctions(_p(d), _p(pair), _p(visited), _p(out))
    return out


MINOR_NAMES = ("A", "B", "Bstar", "D")


def minor(dims, pair, s1, junc, s2):
    """COO (rows, cols, multiplicity) of A (1s x j), B (j x j), B* (j x 2s), D (1s x 2s)."""
    d = _dims(dims)
    lib = _load()
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    junc = np.ascontiguousarray(junc, dtype=np.uint32)
    s2 = np.ascontiguousarray(s2, dtype=np.uint32)
    h = lib.ora_minor(_p(d), _p(pair), len(s1), _p(s1), len(junc), _p(junc), len(s2), _p(s2))
    out = {}
    try:
        st = lib.ora_minor_status(h)
        if st:
            raise OracleError(st, "minor")
        for which, name in enumerate(MINOR_NAMES):
            n = lib.ora_minor_size(h, which)
            rows = np.empty(n, dtype=np.uint32)
            cols = np.empty(n, dtype=np.uint32)
            mult = np.empty(n, dtype=np.uint64)
            if n:
                lib.ora_minor_copy(h, which, _p(rows), _p(cols), _p(mult))
            out[name] = (rows, cols, mult)
    finally:
        lib.ora_minor_free(h)
    return out


def path_counts(dims, pair, s1, s2, src_ranks=None):
    """D* entries (row = 1-saddle rank, col = 2-saddle rank, uint64 count), sorted by (row, col)."""
    d = _dims(dims)
    lib = _load()
    s1 = np.ascontiguousarray(s1, dtype=np.uint32)
    s2 = np.ascontiguousarray(s2, dtype=np.uint32)
    src = None if src_ranks is None else np.ascontiguousarray(src_ranks, dtype=np.int64)
    h = lib.ora_path_counts(_p(d), _p(pair), len(s1), _p(s1), len(s2), _p(s2),
                            0 if src is None else len(src), _p(src))
    try:
        st = lib.ora_result_status(h)
        if st:
            raise OracleError(st, "path_counts")
        n = lib.ora_result_size(h)
        rows = np.empty(n, dtype=np.uint32)
        cols = np.empty(n, dtype=np.uint32)
        cnt = np.empty(n, dtype=np.uint64)
        if n:
            lib.ora_result_copy(h, _p(rows), _p(cols), _p(cnt))
        return rows, cols, cnt
    finally:
        lib.ora_result_free(h)


def n_iter(nj, A, B):
    acols = np.ascontiguousarray(A[1], dtype=np.uint32)
    brows = np.ascontiguousarray(B[0], dtype=np.uint32)
    bcols = np.ascontiguousarray(B[1], dtype=np.uint32)
    return int(_load().ora_n_iter(int(nj), len(acols), _p(acols), len(brows), _p(brows), _p(bcols)))


def compute_all(f: np.ndarray, with_minor: bool = True, with_dstar: bool = True) -> dict:
    """Every output of the pipeline for one field (small and medium grids)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    d = _dims(f)
    pair = gradient(f)
    counts, lists = critical(d, pair)
    vmin, cmax, amin, amax = extremum(d, pair, lists[1], lists[2])
    vis, levels = reachable(d, pair)
    junc = junctions(d, pair, vis)
    res = dict(dims=d, pair=pair, packed=pack(d, pair), counts=counts, lists=lists, vertex_min=vmin,
               cube_max=cmax, min_arcs=amin, max_arcs=amax, visited=vis, levels=levels, junctions=junc)
    if with_minor:
        mn = minor(d, pair, lists[1], junc, lists[2])
        res["minor"] = mn
        res["n_iter"] = n_iter(len(junc), mn["A"], mn["B"])
    if with_dstar:
        res["dstar"] = path_counts(d, pair, lists[1], lists[2])
    return res


def complex_graph(counts, lists, min_arcs, max_arcs, dstar):
    """The 1-skeleton as one adjacency with every arc at both ends (Sec. 3.5 "Data structure").

    Nodes: the critical cells, minima, then 1-saddles, 2-saddles, maxima, each group in cell-id
    order.  Arcs: each 1-saddle's two arcs to minima and each 2-saddle's two arcs to maxima (an
    arc to NONE, which leaves the domain, is left out), one unit each; each D* entry (1-saddle,
    2-saddle, count) as `count` arcs.  Returns (nodeptr, adj, mult): node u's neighbours in
    increasing order, each with the number of arcs joining the two."""
    c = [int(x) for x in counts]
    base = np.cumsum([0] + c)
    us, vs, ms = [], [], []

    def add(u, v, m):  # both directions
        us.extend([u, v])
        vs.extend([v, u])
        ms.extend([m, m])

    s1 = np.repeat(np.arange(c[1], dtype=np.int64), 2)
    add(base[1] + s1, base[0] + np.searchsorted(lists[0], np.asarray(min_arcs[:2 * c[1]])), np.ones(2 * c[1], np.uint64))
    ma = np.asarray(max_arcs[:2 * c[2]])
    keep = ma != NONE
    s2 = np.repeat(np.arange(c[2], dtype=np.int64), 2)[keep]
    add(base[2] + s2, base[3] + np.searchsorted(lists[3], ma[keep]), np.ones(int(keep.sum()), np.uint64))
    rows, cols, cnt = dstar
    add(base[1] + np.asarray(rows, np.int64), base[2] + np.asarray(cols, np.int64), np.asarray(cnt, np.uint64))
    u = np.concatenate([np.asarray(x, np.int64) for x in us]) if us else np.zeros(0, np.int64)
    v = np.concatenate([np.asarray(x, np.int64) for x in vs]) if vs else np.zeros(0, np.int64)
    m = np.concatenate([np.asarray(x, np.uint64) for x in ms]) if ms else np.zeros(0, np.uint64)
    n = int(base[4])
    key = u * max(n, 1) + v
    uniq, first = np.unique(key, return_index=True)
    order = np.argsort(key, kind="stable")
    sums = np.add.reduceat(m[order], np.searchsorted(key[order], uniq)) if len(uniq) else np.zeros(0, np.uint64)
    uu, vv = uniq // max(n, 1), uniq % max(n, 1)
    nodeptr = np.zeros(n + 1, np.int64)
    np.add.at(nodeptr, uu + 1, 1)
    return np.cumsum(nodeptr), vv.astype(np.uint32), sums.astype(np.uint64)


def cell_values(f: np.ndarray, cells) -> np.ndarray:
    """Value of each cell (reading S1 of the simplification): the value of its highest vertex."""
    nz, ny, nx = f.shape
    rx, ry = 2 * nx - 1, 2 * ny - 1
    c = np.asarray(cells, dtype=np.int64)
    cx, cy, cz = c % rx, (c // rx) % ry, c // (rx * ry)
    flat = np.ascontiguousarray(f, dtype=np.float32).reshape(-1)
    best = np.full(len(c), -np.inf)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                x, y, z = (cx + dx * (cx & 1)) // 2, (cy + dy * (cy & 1)) // 2, (cz + dz * (cz & 1)) // 2
                best = np.maximum(best, flat[x + nx * (y + ny * z)].astype(np.float64))
    return best


def skeleton(f: np.ndarray, e: dict | None = None) -> dict:
    """The 1-skeleton of f as simplification input: nodes (critical cells numbered minima,
    1-saddles, 2-saddles, maxima) with index, cell id and value, and arcs (u < v) with their
    multiplicity (complex_graph's adjacency)."""
    e = e or compute_all(f, with_minor=False)
    counts, lists = e["counts"], e["lists"]
    nodeptr, adj, mult = complex_graph(counts, lists, e["min_arcs"], e["max_arcs"], e["dstar"])
    index = np.concatenate([np.full(int(counts[k]), k, np.int32) for k in range(4)])
    cells = np.concatenate([np.asarray(lists[k], np.uint32) for k in range(4)])
    u = np.repeat(np.arange(len(nodeptr) - 1, dtype=np.int64), np.diff(nodeptr))
    keep = u < adj
    return dict(index=index, cell=cells, value=cell_values(f, cells), arc_u=u[keep].astype(np.uint32),
                arc_v=adj[keep].astype(np.uint32), arc_mult=mult[keep].astype(np.uint64))


def simplify(sk: dict, threshold: float, rounds: bool = False) -> dict:
    """Persistence-ordered cancellation of the skeleton's single-arc pairs up to `threshold`
    (Sec. 4; readings S1-S4 in the source).  Returns the cancellation log (upper node, lower node,
    persistence, in order), the surviving nodes and the surviving arcs (u < v, multiplicity).
    rounds=True: in rounds of independent cancellations (reading S5), with each cancellation's
    round in "round" and the number of rounds in "n_rounds"."""
    n = len(sk["index"])
    index = np.ascontiguousarray(sk["index"], np.int32)
    value = np.ascontiguousarray(sk["value"], np.float64)
    cell = np.ascontiguousarray(sk["cell"], np.uint32)
    au = np.ascontiguousarray(sk["arc_u"], np.uint32)
    av = np.ascontiguousarray(sk["arc_v"], np.uint32)
    am = np.ascontiguousarray(sk["arc_mult"], np.uint64)
    lib = _load()
    fn = lib.ora_simplify_rounds if rounds else lib.ora_simplify
    h = fn(n, _p(index), _p(value), _p(cell), len(au), _p(au), _p(av), _p(am), float(threshold))
    extra = {}
    try:
        st = lib.ora_simplify_status(h)
        if st:
            raise OracleError(st, "simplify")
        k, m = lib.ora_simplify_cancelled(h), lib.ora_simplify_arcs(h)
        up, lo, pers = np.empty(k, np.uint32), np.empty(k, np.uint32), np.empty(k, np.float64)
        alive = np.empty(n, np.uint8)
        u, v, mult = np.empty(m, np.uint32), np.empty(m, np.uint32), np.empty(m, np.uint64)
        lib.ora_simplify_copy(h, _p(up), _p(lo), _p(pers), _p(alive), _p(u), _p(v), _p(mult))
        if rounds:
            rnd = np.empty(k, np.uint32)
            lib.ora_simplify_rounds_of(h, _p(rnd))
            extra = dict(round=rnd, n_rounds=int(lib.ora_simplify_rounds_count(h)))
    finally:
        lib.ora_simplify_free(h)
    return dict(upper=up, lower=lo, persistence=pers, alive=alive.astype(bool), arc_u=u, arc_v=v, arc_mult=mult,
                **extra)


# ---- sampled queries on large volumes (pairs computed lazily, one lower star at a time) ----
def lazy_pairs(f, cells):
    f = np.ascontiguousarray(f, dtype=np.float32)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    out = np.empty(len(cells), dtype=np.uint32)
    st = _load().ora_lazy_pairs(_p(_dims(f)), _p(f), len(cells), _p(cells), _p(out))
    if st:
        raise OracleError(st, "lazy_pairs")
    return out


def lazy_vertex_min(f, verts):
    f = np.ascontiguousarray(f, dtype=np.float32)
    verts = np.ascontiguousarray(verts, dtype=np.int64)
    out = np.empty(len(verts), dtype=np.uint32)
    st = _load().ora_lazy_vertex_min(_p(_dims(f)), _p(f), len(verts), _p(verts), _p(out))
    if st:
        raise OracleError(st, "lazy_vertex_min")
    return out


def lazy_cube_max(f, verts):
    f = np.ascontiguousarray(f, dtype=np.float32)
    verts = np.ascontiguousarray(verts, dtype=np.int64)
    out = np.empty(len(verts), dtype=np.uint32)
    st = _load().ora_lazy_cube_max(_p(_dims(f)), _p(f), len(verts), _p(verts), _p(out))
    if st:
        raise OracleError(st, "lazy_cube_max")
    return out


def lazy_nodes(f, cells):
    """(is DAG node, is critical, out-degree) of each listed 1-cell."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    out = np.empty((len(cells), 3), dtype=np.int32)
    st = _load().ora_lazy_nodes(_p(_dims(f)), _p(f), len(cells), _p(cells), _p(out))
    if st:
        raise OracleError(st, "lazy_nodes")
    return out


def lazy_dstar_rows(f, s1_cells):
    """{1-saddle cell: {2-saddle cell: count}} for the listed 1-saddles."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    cells = np.ascontiguousarray(s1_cells, dtype=np.uint32)
    lib = _load()
    h = lib.ora_lazy_dstar_rows(_p(_dims(f)), _p(f), len(cells), _p(cells))
    try:
        st = lib.ora_result_status(h)
        if st:
            raise OracleError(st, "lazy_dstar_rows")
        n = lib.ora_result_size(h)
        rows = np.empty(n, dtype=np.uint32)
        cols = np.empty(n, dtype=np.uint32)
        cnt = np.empty(n, dtype=np.uint64)
        if n:
            lib.ora_result_copy(h, _p(rows), _p(cols), _p(cnt))
    finally:
        lib.ora_result_free(h)
    out = {int(c): {} for c in cells}
    for r, c, k in zip(rows, cols, cnt):
        out[int(cells[r])][int(c)] = int(k)
    return out
