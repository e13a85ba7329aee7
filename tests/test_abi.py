"""CPU-side checks of the C ABI: the library builds, loads, and exports every symbol that
include/msc.h declares (no compute calls: there may be no GPU)."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:msc_status|const char\*)\s+(msc_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2009_03707_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 13
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2009_03707_gb300 import msc

    assert _declared() <= set(msc.SIGNATURES)


def test_plan_frees_every_buffer_exactly_once():
    """msc_plan_destroy frees the buffers that Plan::for_each_buffer lists: each declared
    DeviceBuffer must appear there exactly once (a repeat would be freed twice, a gap leaked)."""
    import collections

    src = open(os.path.join(ROOT, "paper_2009_03707_gb300", "csrc", "msc_internal.cuh")).read()
    decl = src[src.index("struct Plan {"):src.index("template <class F>")]
    declared = []
    for line in decl.splitlines():
        line = line.strip()
        if not line.startswith("DeviceBuffer "):
            continue
        for item in line[len("DeviceBuffer "):].rstrip(";").split(","):
            m = re.match(r"\s*(\w+)(?:\[(\d+)\])?", item)
            name, n = m.group(1), m.group(2)
            declared += [f"{name}[{i}]" for i in range(int(n))] if n else [name]
    block = src[src.index("DeviceBuffer* all[] = {"):src.index("for (DeviceBuffer* b : all)")]
    listed = re.findall(r"&(\w+(?:\[\d+\])?)", block)
    assert [n for n, c in collections.Counter(listed).items() if c > 1] == []
    assert sorted(listed) == sorted(declared)


def test_plan_rejects_unknown_options_before_touching_the_device():
    """msc_plan checks its options first: unknown flag bits and out-of-range selectors are
    MSC_ERR_ARG with no plan made (so this runs without a GPU)."""
    from paper_2009_03707_gb300 import build, msc

    lib = ctypes.CDLL(build.build())
    lib.msc_plan.restype = ctypes.c_int
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    known = msc.MSC_FLAG_NO_GRAPH | msc.MSC_FLAG_SERIAL_PASS
    for flags, tile, method in [(4, 0, 0), (known | 8, 0, 0), (0, 10, 0), (0, -1, 0), (0, 0, 3)]:
        opts = msc.MscOpts(0, flags, 0, tile, method)
        out = ctypes.c_void_p(1)
        assert lib.msc_plan(dims, ctypes.byref(opts), ctypes.byref(out)) == 1
        assert not out.value


def test_binding_flag_values_match_the_header():
    """Every MSC_FLAG_* the header defines has the same value in the binding."""
    from paper_2009_03707_gb300 import msc

    text = open(os.path.join(ROOT, "include", "msc.h")).read()
    flags = dict(re.findall(r"^#define\s+(MSC_FLAG_\w+)\s+(\d+)", text, re.M))
    assert {"MSC_FLAG_NO_GRAPH", "MSC_FLAG_SERIAL_PASS"} <= set(flags)
    for name, value in flags.items():
        assert getattr(msc, name) == int(value), name
