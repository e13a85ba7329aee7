"""msc_copy_to_host: every output of a pass copied into caller-owned host memory, equal to the
device arrays the accessors return, with the size query, the capacity error and argument checks;
on a field whose stages have not run yet, the copy runs them (and the result is the oracle's)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from synth import fields
from tests.gpu_util import dims_of, gpu_field, msc, to_np

pytestmark = pytest.mark.gpu


def test_every_output_equals_the_device_arrays():
    m = msc()
    f = fields.grf((40, 36, 33), 3.0, seed=81)
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    counts, cells = m.msc_critical(plan)
    amin, amax, vmin, cmax = m.msc_extremum_arcs(plan)
    rowptr, col, cnt = m.msc_saddle_arcs(plan)
    want = {"cells0": cells[0], "cells1": cells[1], "cells2": cells[2], "cells3": cells[3], "min_arcs": amin,
            "max_arcs": amax, "vertex_min": vmin, "cube_max": cmax, "dstar_rowptr": rowptr, "dstar_col": col,
            "dstar_count": cnt}
    for name, dev in want.items():
        got = m.msc_copy_to_host(plan, name)
        assert np.array_equal(got, to_np(dev).reshape(-1)), name


def test_copy_runs_the_stages():
    m = msc()
    f = fields.grf((20, 22, 24), 3.0, seed=82)
    plan = m.Plan(dims_of(f))
    m.msc_gradient(plan, gpu_field(f))   # only the gradient so far
    e = oracle.compute_all(f, with_minor=False, with_dstar=True)
    assert np.array_equal(m.msc_copy_to_host(plan, "cells2"), e["lists"][2])
    assert np.array_equal(m.msc_copy_to_host(plan, "min_arcs"), e["min_arcs"])
    rows, cols, cnt = e["dstar"]
    assert np.array_equal(m.msc_copy_to_host(plan, "dstar_col"), cols)
    assert np.array_equal(m.msc_copy_to_host(plan, "dstar_count"), cnt)


def test_size_query_capacity_and_arguments():
    m = msc()
    f = fields.grf((16, 16, 16), 3.0, seed=83)
    plan = m.Plan(dims_of(f))
    m.msc_compute(plan, gpu_field(f))
    lib = m.lib
    n = ctypes.c_int64(0)
    assert lib.msc_copy_to_host(plan.handle, None, 6, None, ctypes.byref(n)) == 0
    assert n.value == 4 * 16 ** 3
    buf = np.zeros(16 ** 3, np.uint32)
    small = ctypes.c_int64(n.value - 4)
    assert lib.msc_copy_to_host(plan.handle, None, 6, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(small)) == 12
    assert small.value == n.value and not buf.any()
    bad = ctypes.c_int64(0)
    assert lib.msc_copy_to_host(plan.handle, None, 15, None, ctypes.byref(bad)) == 1  # past the last selector
    assert lib.msc_copy_to_host(plan.handle, None, -1, None, ctypes.byref(bad)) == 1


def test_every_query_before_a_pass_is_a_state_error():
    """On a plan that has seen no field, every stage query, on-request output and host copy returns
    MSC_ERR_STATE (nothing runs), and the plan then computes normally."""
    m = msc()
    f = fields.grf((14, 15, 16), 3.0, seed=85)
    plan = m.Plan(dims_of(f))
    d = gpu_field(f)
    calls = [lambda: m.msc_critical(plan), lambda: m.msc_extremum_arcs(plan), lambda: m.msc_saddle_arcs(plan),
             lambda: m.msc_saddle_arcs_csc(plan), lambda: m.msc_arc_geometry(plan),
             lambda: m.msc_saddle_arc_geometry(plan), lambda: m.msc_complex_graph(plan),
             lambda: m.msc_simplify(plan, d, 0.1)]
    calls += [lambda w=w: m.msc_copy_to_host(plan, w) for w in m.MSC_OUT]
    for call in calls:
        with pytest.raises(m.MscError) as err:
            call()
        assert err.value.status == 11  # MSC_ERR_STATE
    m.msc_compute(plan, d)
    e = oracle.compute_all(f)
    counts, _ = m.msc_critical(plan)
    assert list(counts) == [len(c) for c in e["lists"]]
    off, cells = m.msc_saddle_arc_geometry(plan)
    want_off, want_cells = oracle.ss_arc_cells(dims_of(f), e["pair"], e["lists"][1], e["lists"][2], e["dstar"])
    assert np.array_equal(to_np(off), want_off) and np.array_equal(to_np(cells), want_cells)
