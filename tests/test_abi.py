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
