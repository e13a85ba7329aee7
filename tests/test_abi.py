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
