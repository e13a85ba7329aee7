"""Thin Python binding of libmsc (include/msc.h): argument marshalling only.

Every function has the name of the C entry point it wraps and passes torch device
pointers and the current CUDA stream straight through; all pipeline arithmetic runs in
the library's CUDA kernels.  Plan-owned outputs are returned as zero-copy torch views
(``__cuda_array_interface__``) that stay valid until the next ``msc_gradient`` on the
same plan or its destruction -- clone them to keep them longer.  There is no CPU path:
if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

MSC_OK = 0
STATUS_NAMES = {0: "MSC_OK", 1: "MSC_ERR_ARG", 2: "MSC_ERR_NAN", 3: "MSC_ERR_OOM", 4: "MSC_ERR_TOO_LARGE",
                6: "MSC_ERR_OVERFLOW", 7: "MSC_ERR_ITER_LIMIT", 8: "MSC_ERR_TIMEOUT", 9: "MSC_ERR_CUDA",
                10: "MSC_NOT_READY", 11: "MSC_ERR_STATE", 12: "MSC_ERR_CAPACITY", 13: "MSC_ERR_INTERNAL"}
MSC_ERR_CAPACITY = 12
MSC_ERR_INTERNAL = 13
MSC_STATIC_SCRATCH_BYTES = 16 << 20

# Every symbol declared in include/msc.h with its ctypes signature.
_P, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)
_PI64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "msc_plan": ([_PI64, _P, _PP], _I32),
    "msc_plan_destroy": ([_P], _I32),
    "msc_last_error_string": ([_P], ctypes.c_char_p),
    "msc_gradient": ([_P, _P, _P], _I32),
    "msc_gradient_words": ([_P, _PP], _I32),
    "msc_critical": ([_P, _P, _PI64, _PP], _I32),
    "msc_extremum_arcs": ([_P, _P, _PP, _PP, _PP, _PP], _I32),
    "msc_reachability": ([_P, _P, _PP, _PI64, _PI64], _I32),
    "msc_junctions": ([_P, _P, _PP, _PI64], _I32),
    "msc_minor": ([_P, _P, _I32, _PI64, _PI64, _PP, _PP, _PP], _I32),
    "msc_saddle_arcs": ([_P, _P, _PI64, _PP, _PP, _PP], _I32),
    "msc_saddle_arcs_csc": ([_P, _P, _PI64, _PP, _PP, _PP], _I32),
    "msc_complex_graph": ([_P, _P, _PI64, _PI64, _P, _P, _P], _I32),
    "msc_arc_geometry": ([_P, _P, _PI64, _PI64, _PP, _PP], _I32),
    "msc_saddle_arc_geometry": ([_P, _P, _PI64, _PI64, _PP, _PP], _I32),
    "msc_simplify": ([_P, _P, _P, ctypes.c_double, _P], _I32),
    "msc_compute_async": ([_P, _P, _P], _I32),
    "msc_copy_to_host": ([_P, _P, _I32, _P, _PI64], _I32),
    "msc_compute_wait": ([_P], _I32),
    "msc_compute": ([_P, _P, _P], _I32),
    "msc_get_stats": ([_P, _P], _I32),
    "msc_static_prepare": ([_I32], _I32),
    "msc_gradient_critical_static": ([_PI64, _P, _P, _PP, _PI64, _PI64, _P], _I32),
    "msc_batch_create": ([_I32, _I64, _PP], _I32),
    "msc_batch_destroy": ([_P], _I32),
    "msc_batch_submit": ([_P, _P, _I32, _P, ctypes.POINTER(ctypes.c_uint64)], _I32),
    "msc_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(_I32), ctypes.POINTER(_I32)], _I32),
    "msc_batch_wait": ([_P, ctypes.c_uint64, ctypes.POINTER(_I32)], _I32),
}


MSC_FLAG_NO_GRAPH = 1
MSC_FLAG_SERIAL_PASS = 2


class MscOpts(ctypes.Structure):
    _fields_ = [("max_iterations", ctypes.c_int64), ("flags", ctypes.c_int32), ("path_count_tier", ctypes.c_int32),
                ("gradient_tile", ctypes.c_int32), ("path_count_method", ctypes.c_int32)]


class MscStats(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_int64 * 4), ("n_reachable", ctypes.c_int64), ("n_bfs_levels", ctypes.c_int64),
                ("n_junctions", ctypes.c_int64), ("nnz_A", ctypes.c_int64), ("nnz_B", ctypes.c_int64),
                ("nnz_Bstar", ctypes.c_int64), ("nnz_D", ctypes.c_int64), ("nnz_Dstar", ctypes.c_int64),
                ("n_iter", ctypes.c_int64), ("n_pointer_jumps", ctypes.c_int64),
                ("max_path_count", ctypes.c_uint64), ("peak_device_bytes", ctypes.c_int64),
                ("n_launches", ctypes.c_int64),
                ("ms_gradient", ctypes.c_float), ("ms_critical", ctypes.c_float), ("ms_extremum", ctypes.c_float),
                ("ms_reachability", ctypes.c_float), ("ms_minor", ctypes.c_float),
                ("ms_path_count", ctypes.c_float), ("ms_rows_kernel", ctypes.c_float),
                ("ms_trace_kernel", ctypes.c_float), ("n_frontier_entries", ctypes.c_int64),
                ("gradient_tile", ctypes.c_int64), ("path_count_method", ctypes.c_int64),
                ("ms_gradient_kernel", ctypes.c_float), ("reserved_f", ctypes.c_float)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["counts"] = list(self.counts)
        return d


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libmsc.so is not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


class MscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, plan=None, what=""):
    if st != MSC_OK:
        msg = lib.msc_last_error_string(plan).decode() if plan else what
        raise MscError(st, msg or what)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _DevArray:
    """Zero-copy view of a plan-owned device buffer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def _view(ptr, shape, typestr):
    n = 1
    for s in shape:
        n *= int(s)
    if n == 0 or not ptr:
        dt = {"<u4": torch.uint32, "<u8": torch.uint64, "<i8": torch.int64, "|u1": torch.uint8}[typestr]
        return torch.empty(tuple(int(s) for s in shape), dtype=dt, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


class Plan:
    """Owns an msc_plan_t for one grid shape (nx, ny, nz)."""

    def __init__(self, dims, max_iterations: int = 0, path_count_tier: int = 0, no_graph: bool = False,
                 gradient_tile: int = 0, path_count_method: int = 0, serial_pass: bool = False):
        self.dims = tuple(int(d) for d in dims)
        arr = (ctypes.c_int64 * 3)(*self.dims)
        flags = (MSC_FLAG_NO_GRAPH if no_graph else 0) | (MSC_FLAG_SERIAL_PASS if serial_pass else 0)
        opts = MscOpts(int(max_iterations), flags, int(path_count_tier),
                       int(gradient_tile), int(path_count_method))
        h = ctypes.c_void_p()
        _check(lib.msc_plan(arr, ctypes.byref(opts), ctypes.byref(h)), what=f"msc_plan{self.dims}")
        self.handle = h

    @classmethod
    def adopt(cls, handle: int, dims):
        """Wrap (and take ownership of) a plan the library created, e.g. by msc_batch_submit."""
        obj = cls.__new__(cls)
        obj.dims = tuple(int(d) for d in dims)
        obj.handle = ctypes.c_void_p(handle)
        return obj

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib.msc_plan_destroy(h)
            self.handle = None

    @property
    def shape_zyx(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)


# ---- the C entry points, by name ---------------------------------------------------------
def msc_plan(dims) -> Plan:
    return Plan(dims)


def msc_gradient(plan: Plan, field: torch.Tensor) -> None:
    if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    if tuple(field.shape) != plan.shape_zyx:
        raise ValueError(f"field shape {tuple(field.shape)} does not match the plan {plan.shape_zyx}")
    _check(lib.msc_gradient(plan.handle, ctypes.c_void_p(field.data_ptr()), _stream()), plan.handle)


def msc_gradient_words(plan: Plan) -> torch.Tensor:
    p = ctypes.c_void_p()
    _check(lib.msc_gradient_words(plan.handle, ctypes.byref(p)), plan.handle)
    return _view(p.value, plan.shape_zyx, "<u4")


def msc_critical(plan: Plan):
    counts = (ctypes.c_int64 * 4)()
    cells = (ctypes.c_void_p * 4)()
    _check(lib.msc_critical(plan.handle, _stream(), counts, cells), plan.handle)
    return [int(c) for c in counts], [_view(cells[k], (counts[k],), "<u4") for k in range(4)]


def msc_extremum_arcs(plan: Plan):
    out = [ctypes.c_void_p() for _ in range(4)]
    _check(lib.msc_extremum_arcs(plan.handle, _stream(), *[ctypes.byref(o) for o in out]), plan.handle)
    counts, _ = msc_critical(plan)
    return (_view(out[0].value, (2 * counts[1],), "<u4"), _view(out[1].value, (2 * counts[2],), "<u4"),
            _view(out[2].value, plan.shape_zyx, "<u4"), _view(out[3].value, plan.shape_zyx, "<u4"))


def msc_reachability(plan: Plan):
    p = ctypes.c_void_p()
    nw = ctypes.c_int64()
    lv = ctypes.c_int64()
    _check(lib.msc_reachability(plan.handle, _stream(), ctypes.byref(p), ctypes.byref(nw), ctypes.byref(lv)),
           plan.handle)
    return _view(p.value, (nw.value,), "<u4"), int(lv.value)


def msc_junctions(plan: Plan):
    p = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(lib.msc_junctions(plan.handle, _stream(), ctypes.byref(p), ctypes.byref(n)), plan.handle)
    return _view(p.value, (n.value,), "<u4")


def msc_minor(plan: Plan, which: int):
    rows, nnz = ctypes.c_int64(), ctypes.c_int64()
    rp, col, mult = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.msc_minor(plan.handle, _stream(), which, ctypes.byref(rows), ctypes.byref(nnz), ctypes.byref(rp),
                         ctypes.byref(col), ctypes.byref(mult)), plan.handle)
    return (_view(rp.value, (rows.value + 1,), "<i8"), _view(col.value, (nnz.value,), "<u4"),
            _view(mult.value, (nnz.value,), "<u4"))


def msc_saddle_arcs(plan: Plan):
    nnz = ctypes.c_int64()
    rp, col, cnt = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.msc_saddle_arcs(plan.handle, _stream(), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(col),
                               ctypes.byref(cnt)), plan.handle)
    counts, _ = msc_critical(plan)
    return (_view(rp.value, (counts[1] + 1,), "<i8"), _view(col.value, (nnz.value,), "<u4"),
            _view(cnt.value, (nnz.value,), "<u8"))


def msc_saddle_arcs_csc(plan: Plan):
    """D* by 2-saddle: (colptr [counts[2]+1] int64, row [nnz] uint32, count [nnz] uint64)."""
    nnz = ctypes.c_int64()
    cp, row, cnt = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.msc_saddle_arcs_csc(plan.handle, _stream(), ctypes.byref(nnz), ctypes.byref(cp), ctypes.byref(row),
                                   ctypes.byref(cnt)), plan.handle)
    counts, _ = msc_critical(plan)
    return (_view(cp.value, (counts[2] + 1,), "<i8"), _view(row.value, (nnz.value,), "<u4"),
            _view(cnt.value, (nnz.value,), "<u8"))


def msc_arc_geometry(plan: Plan):
    """The cells along every saddle-extremum arc: (offsets [n_arcs+1] int64, cells [n_cells] uint32),
    arcs numbered as the arc lists (2 per 1-saddle, then 2 per 2-saddle)."""
    n_arcs, n_cells = ctypes.c_int64(), ctypes.c_int64()
    off, cells = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.msc_arc_geometry(plan.handle, _stream(), ctypes.byref(n_arcs), ctypes.byref(n_cells), ctypes.byref(off),
                                ctypes.byref(cells)), plan.handle)
    return _view(off.value, (n_arcs.value + 1,), "<i8"), _view(cells.value, (n_cells.value,), "<u4")


def msc_saddle_arc_geometry(plan: Plan):
    """The cells along every saddle-saddle arc of multiplicity 1: (offsets [nnz+1] int64, cells
    [n_cells] uint32), one range per D* entry in msc_saddle_arcs order (empty when its count is not 1)."""
    nnz, n_cells = ctypes.c_int64(), ctypes.c_int64()
    off, cells = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.msc_saddle_arc_geometry(plan.handle, _stream(), ctypes.byref(nnz), ctypes.byref(n_cells),
                                       ctypes.byref(off), ctypes.byref(cells)), plan.handle)
    return _view(off.value, (nnz.value + 1,), "<i8"), _view(cells.value, (n_cells.value,), "<u4")


class MscSimplified(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_rounds", ctypes.c_int64), ("n_cancelled", ctypes.c_int64),
                ("n_adj", ctypes.c_int64), ("counts", ctypes.c_int64 * 4), ("d_alive", ctypes.c_void_p),
                ("d_nodeptr", ctypes.c_void_p), ("d_adj", ctypes.c_void_p), ("d_mult", ctypes.c_void_p),
                ("d_log", ctypes.c_void_p)]


def msc_simplify(plan: Plan, field: torch.Tensor, threshold: float) -> dict:
    """Cancels critical-point pairs up to `threshold` (absolute persistence) on the GPU, in rounds of
    independent cancellations; `field` is the plan's last pass's field.  Returns the counts left, the
    rounds, and zero-copy views of the result (alive flags, CSR adjacency, cancellation log)."""
    if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    if tuple(field.shape) != plan.shape_zyx:
        raise ValueError(f"field shape {tuple(field.shape)} does not match the plan {plan.shape_zyx}")
    o = MscSimplified()
    _check(lib.msc_simplify(plan.handle, _stream(), ctypes.c_void_p(field.data_ptr()), float(threshold),
                            ctypes.byref(o)), plan.handle)
    n, nadj, k = o.n_nodes, o.n_adj, o.n_cancelled
    return dict(counts=[int(c) for c in o.counts], n_rounds=int(o.n_rounds), n_cancelled=int(k),
                alive=_view(o.d_alive, (n,), "|u1"), nodeptr=_view(o.d_nodeptr, (n + 1,), "<i8"),
                adj=_view(o.d_adj, (nadj,), "<u4"), mult=_view(o.d_mult, (nadj,), "<u8"),
                log=_view(o.d_log, (k, 3), "<u4"))


def msc_complex_graph(plan: Plan):
    """The 1-skeleton on the host: (nodeptr [n_nodes+1] int64, adj [n_adj] uint32, mult [n_adj]
    uint64) over nodes numbered minima, 1-saddles, 2-saddles, maxima."""
    n_nodes, n_adj = ctypes.c_int64(), ctypes.c_int64(0)
    _check(lib.msc_complex_graph(plan.handle, _stream(), ctypes.byref(n_nodes), ctypes.byref(n_adj), None, None, None),
           plan.handle)
    nodeptr = np.empty(n_nodes.value + 1, dtype=np.int64)  # every entry is written by the copy
    adj = np.empty(max(n_adj.value, 1), dtype=np.uint32)
    mult = np.empty(max(n_adj.value, 1), dtype=np.uint64)
    _check(lib.msc_complex_graph(plan.handle, _stream(), ctypes.byref(n_nodes), ctypes.byref(n_adj),
                                 nodeptr.ctypes.data_as(ctypes.c_void_p), adj.ctypes.data_as(ctypes.c_void_p),
                                 mult.ctypes.data_as(ctypes.c_void_p)), plan.handle)
    return nodeptr, adj[:n_adj.value], mult[:n_adj.value]


def msc_complex_graph_size(plan: Plan):
    """Builds the 1-skeleton on the device if needed and returns (n_nodes, n_adj), copying nothing."""
    n_nodes, n_adj = ctypes.c_int64(), ctypes.c_int64(0)
    _check(lib.msc_complex_graph(plan.handle, _stream(), ctypes.byref(n_nodes), ctypes.byref(n_adj), None, None, None),
           plan.handle)
    return int(n_nodes.value), int(n_adj.value)


def msc_compute(plan: Plan, field: torch.Tensor) -> None:
    if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    if tuple(field.shape) != plan.shape_zyx:
        raise ValueError(f"field shape {tuple(field.shape)} does not match the plan {plan.shape_zyx}")
    _check(lib.msc_compute(plan.handle, ctypes.c_void_p(field.data_ptr()), _stream()), plan.handle)


MSC_OUT = {"cells0": (0, np.uint32), "cells1": (1, np.uint32), "cells2": (2, np.uint32), "cells3": (3, np.uint32),
           "min_arcs": (4, np.uint32), "max_arcs": (5, np.uint32), "vertex_min": (6, np.uint32),
           "cube_max": (7, np.uint32), "dstar_rowptr": (8, np.int64), "dstar_col": (9, np.uint32),
           "dstar_count": (10, np.uint64), "arc_offsets": (11, np.int64), "arc_cells": (12, np.uint32),
           "ss_arc_offsets": (13, np.int64), "ss_arc_cells": (14, np.uint32)}


def msc_copy_to_host(plan: Plan, what: str) -> np.ndarray:
    """One output of the last pass as a host numpy array (size query, then the copy)."""
    code, dtype = MSC_OUT[what]
    nbytes = ctypes.c_int64(0)
    _check(lib.msc_copy_to_host(plan.handle, _stream(), code, None, ctypes.byref(nbytes)), plan.handle)
    out = np.empty(nbytes.value // np.dtype(dtype).itemsize, dtype=dtype)
    room = ctypes.c_int64(out.nbytes)
    _check(lib.msc_copy_to_host(plan.handle, _stream(), code, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(room)),
           plan.handle)
    return out


def msc_copy_to_host_size(plan: Plan, what: str) -> int:
    """Size in bytes of one output of the last pass (msc_copy_to_host's size query)."""
    nbytes = ctypes.c_int64(0)
    _check(lib.msc_copy_to_host(plan.handle, _stream(), MSC_OUT[what][0], None, ctypes.byref(nbytes)), plan.handle)
    return int(nbytes.value)


def msc_copy_to_host_into(plan: Plan, what: str, out: torch.Tensor) -> int:
    """Copies one output of the last pass into a caller-owned host tensor (pinned memory for a
    direct DMA); returns the bytes copied.  MSC_ERR_CAPACITY if the tensor is too small."""
    if out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous host tensor")
    room = ctypes.c_int64(out.numel() * out.element_size())
    _check(lib.msc_copy_to_host(plan.handle, _stream(), MSC_OUT[what][0], ctypes.c_void_p(out.data_ptr()),
                                ctypes.byref(room)), plan.handle)
    return int(room.value)


def msc_compute_async(plan: Plan, field: torch.Tensor) -> None:
    """Enqueues the pass on the current stream and returns (see msc_compute_wait)."""
    if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    if tuple(field.shape) != plan.shape_zyx:
        raise ValueError(f"field shape {tuple(field.shape)} does not match the plan {plan.shape_zyx}")
    _check(lib.msc_compute_async(plan.handle, ctypes.c_void_p(field.data_ptr()), _stream()), plan.handle)


def msc_compute_wait(plan: Plan) -> None:
    _check(lib.msc_compute_wait(plan.handle), plan.handle)


def msc_get_stats(plan: Plan) -> dict:
    s = MscStats()
    _check(lib.msc_get_stats(plan.handle, ctypes.byref(s)), plan.handle)
    return s.as_dict()


def diagnostics(stats: dict) -> dict:
    """The statistics of the paper's performance analysis (Sec. 4.2) from a run's msc_get_stats:
    critical points, saddles and junction nodes (and junctions per critical point), the sparsity
    ratio (zero entries / all entries) of A (1-saddles x junctions), B (junctions x junctions),
    B* (junctions x 2-saddles), D and D* (1-saddles x 2-saddles), and the number of iterations of
    the product loop.  A ratio is None for a matrix with no rows or no columns."""
    c = [int(x) for x in stats["counts"]]
    n1, n2, nj = c[1], c[2], int(stats["n_junctions"])
    ncrit = sum(c)

    def sparsity(nnz, rows, cols):
        return None if rows * cols == 0 else 1.0 - int(nnz) / (rows * cols)

    return dict(critical=ncrit, saddles=n1 + n2, extrema=c[0] + c[3], junctions=nj,
                junctions_per_critical=None if ncrit == 0 else nj / ncrit,
                sparsity=dict(A=sparsity(stats["nnz_A"], n1, nj), B=sparsity(stats["nnz_B"], nj, nj),
                              Bstar=sparsity(stats["nnz_Bstar"], nj, n2), D=sparsity(stats["nnz_D"], n1, n2),
                              Dstar=sparsity(stats["nnz_Dstar"], n1, n2)),
                n_iter=int(stats["n_iter"]), max_path_count=int(stats["max_path_count"]),
                bfs_levels=int(stats["n_bfs_levels"]), peak_device_bytes=int(stats["peak_device_bytes"]))


def msc_gradient_critical_static(field: torch.Tensor, words: torch.Tensor, cells, capacity) -> list:
    """Stages (a1)+(a2) into caller-owned tensors with no device allocation by the library.

    For callers that cannot allocate device memory (the GPU's memory already belongs to their
    own pool, or they run inside a callback or deadline-bound loop where cudaMalloc is not
    allowed).  field: [nz,ny,nx] float32; words: [nz,ny,nx] uint32 output; cells: 4 uint32
    output tensors; capacity: their entry capacities.  Returns the 4 critical counts.  Scratch
    lives in one static device array shared by every call, so overlapping calls race.
    """
    if field.dtype != torch.float32 or not field.is_cuda or not field.is_contiguous() or field.dim() != 3:
        raise ValueError("field must be a contiguous 3-D float32 CUDA tensor")
    dev = field.device
    if dev.index != torch.cuda.current_device():
        raise ValueError(f"field is on {dev}, but the current device is cuda:{torch.cuda.current_device()}")
    nz, ny, nx = field.shape
    if (tuple(words.shape) != (nz, ny, nx) or words.dtype != torch.uint32 or not words.is_contiguous()
            or words.device != dev):
        raise ValueError("words must be a contiguous uint32 tensor shaped like the field, on its device")
    if len(cells) != 4 or len(capacity) != 4:
        raise ValueError("cells and capacity need one entry per cell dimension (4)")
    for k in range(4):
        c, cap_k = cells[k], int(capacity[k])
        if c.dtype != torch.uint32 or not c.is_contiguous() or c.device != dev:
            raise ValueError(f"cells[{k}] must be a contiguous uint32 tensor on {dev}")
        if cap_k < 0 or cap_k > c.numel():
            raise ValueError(f"capacity[{k}] = {cap_k} exceeds cells[{k}].numel() = {c.numel()}")
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    ptrs = (ctypes.c_void_p * 4)(*[c.data_ptr() if c.numel() else None for c in cells])
    cap = (ctypes.c_int64 * 4)(*[int(c) for c in capacity])
    counts = (ctypes.c_int64 * 4)()
    st = lib.msc_gradient_critical_static(dims, ctypes.c_void_p(field.data_ptr()), ctypes.c_void_p(words.data_ptr()),
                                          ptrs, cap, counts, _stream())
    if st != MSC_OK:
        raise MscError(st, f"msc_gradient_critical_static{(nx, ny, nz)} counts={list(counts)}")
    return [int(c) for c in counts]


def msc_static_prepare(device: int) -> None:
    """Loads the library's device code on `device` and looks up the static scratch array of
    msc_gradient_critical_static there, without running anything (call it before the rest of the
    GPU's memory is reserved)."""
    _check(lib.msc_static_prepare(int(device)), what=f"msc_static_prepare({device})")


class MscVolume(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("d_field", ctypes.c_void_p), ("plan", ctypes.c_void_p)]


class Batch:
    """msc_batch_*: a pool of worker threads/streams that runs submitted volumes concurrently,
    admitting them against an HBM budget (continuous batching)."""

    def __init__(self, n_workers: int = 4, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(lib.msc_batch_create(int(n_workers), int(hbm_budget_bytes), ctypes.byref(h)), what="msc_batch_create")
        self.handle = h
        self._inflight = {}

    def msc_batch_submit(self, fields, plans=None):
        """Queue volumes; returns (ticket, plans).  A None plan is created by the library."""
        n = len(fields)
        plans = list(plans) if plans is not None else [None] * n
        vols = (MscVolume * n)()
        for i, f in enumerate(fields):
            if f.dtype != torch.float32 or not f.is_cuda or not f.is_contiguous():
                raise ValueError("fields must be contiguous float32 CUDA tensors")
            nz, ny, nx = f.shape
            vols[i].dims[:] = (nx, ny, nz)
            vols[i].d_field = f.data_ptr()
            vols[i].plan = plans[i].handle.value if plans[i] is not None else None
        t = ctypes.c_uint64()
        _check(lib.msc_batch_submit(self.handle, vols, n, _stream(), ctypes.byref(t)), what="msc_batch_submit")
        out = []
        for i, f in enumerate(fields):
            if plans[i] is None:
                nz, ny, nx = f.shape
                plans[i] = Plan.adopt(vols[i].plan, (nx, ny, nz))
            out.append(plans[i])
        self._inflight[t.value] = (list(fields), out)  # keep inputs and plans alive
        return t.value, out

    def msc_poll(self, ticket: int):
        done, status = ctypes.c_int(), ctypes.c_int()
        _check(lib.msc_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(status)),
               what="msc_poll")
        if done.value:
            self._inflight.pop(ticket, None)
        return bool(done.value), int(status.value)

    def msc_batch_wait(self, ticket: int) -> int:
        status = ctypes.c_int()
        _check(lib.msc_batch_wait(self.handle, ctypes.c_uint64(ticket), ctypes.byref(status)), what="msc_batch_wait")
        self._inflight.pop(ticket, None)
        return int(status.value)

    def close(self):
        if getattr(self, "handle", None):
            lib.msc_batch_destroy(self.handle)
            self.handle = None
            self._inflight.clear()

    def __del__(self):
        self.close()


def compute(field: torch.Tensor, plan: Plan | None = None) -> dict:
    """All outputs of the pipeline for one device field, as torch tensors on its device."""
    nz, ny, nx = field.shape
    plan = plan or Plan((nx, ny, nz))
    msc_compute(plan, field)
    counts, cells = msc_critical(plan)
    min_arcs, max_arcs, vmin, cmax = msc_extremum_arcs(plan)
    rowptr, col, cnt = msc_saddle_arcs(plan)
    return dict(plan=plan, counts=counts, cells=cells, min_arcs=min_arcs, max_arcs=max_arcs, vertex_min=vmin,
                cube_max=cmax, dstar=(rowptr, col, cnt), stats=msc_get_stats(plan))
