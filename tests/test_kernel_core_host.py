"""The per-vertex lower-star core of the CUDA gradient kernel (csrc/lower_star.cuh) is
host+device code; this CPU test compiles it with g++ and checks the packed words it produces
against the oracle, so logic errors surface before any GPU run."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from synth import fields
from tests.cubical import random_field

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("harness") / "liblower_star_host.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                           os.path.join(HERE, "host_harness", "lower_star_host.cpp")])
    lib = ctypes.CDLL(out)
    lib.host_words.argtypes = [ctypes.c_void_p] * 3
    lib.host_words.restype = ctypes.c_int
    return lib


def _cases():
    out = [fields.cosine_lattice(), fields.grf((30, 31, 33), 3.0, seed=4),
           fields.gaussian_blobs(n=24, n_blobs=5, sigma_range=(2, 5), seed=7)]
    for i, shp in enumerate([(2, 2, 2), (3, 5, 7), (9, 8, 33), (6, 6, 6), (4, 3, 2)]):
        out.append(random_field(shp, 40 + i, "normal"))
        out.append(random_field(shp, 60 + i, "ties"))
        out.append(random_field(shp, 80 + i, "near"))
    return out


@pytest.mark.parametrize("f", _cases(), ids=lambda f: "x".join(map(str, f.shape)))
def test_kernel_core_matches_oracle(host_lib, f):
    nz, ny, nx = f.shape
    d = np.array([nx, ny, nz], dtype=np.int64)
    words = np.empty(f.shape, dtype=np.uint32)
    f = np.ascontiguousarray(f, dtype=np.float32)
    bad = host_lib.host_words(d.ctypes.data, f.ctypes.data, words.ctypes.data)
    assert bad == 0
    assert np.array_equal(words, oracle.pack(d, oracle.gradient(f)))


def test_one_free_facet_mask_matches_its_definition(host_lib):
    """The core finds the cells with exactly one unclassified facet for all 27 positions at once
    (shifts by 1, 3 and 9); it must agree with counting each cell's facets one by one."""
    host_lib.host_one_free_facet_mismatches.argtypes = [ctypes.c_int]
    host_lib.host_one_free_facet_mismatches.restype = ctypes.c_int
    assert host_lib.host_one_free_facet_mismatches(200000) == 0


def test_least_edge_by_keys_matches_the_cell_order(host_lib):
    """The core picks x's lowest edge by comparing the edges' vertex keys directly; that must be
    the least edge under the general cell order (vertex lists sorted downwards, ties by index)."""
    host_lib.host_edge_min_mismatches.argtypes = [ctypes.c_int]
    host_lib.host_edge_min_mismatches.restype = ctypes.c_int
    assert host_lib.host_edge_min_mismatches(200000) == 0
