"""The oracle's pins must be able to fail: each test here plants one plausible mistake in a
copy of the oracle's source (on the CPU), rebuilds it, and checks that at least one pin of
tests/test_oracle_pins.py rejects the broken copy.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

# (name, exact text in msc_oracle.cpp, replacement)
MUTANTS = [
    ("tie_break_reversed", "        return a < b;\n    }\n    // Vertices", "        return a > b;\n    }\n    // Vertices"),
    ("pair_vertex_with_greatest_edge",
     "if (ls.cells[i].dim == 1 && (delta < 0 || ls.key_less(i, delta))) delta = i;",
     "if (ls.cells[i].dim == 1 && (delta < 0 || ls.key_less(delta, i))) delta = i;"),
    ("pq_one_no_reinsert_of_partner_cofacets",
     "            nb.insert(nb.end(), nb2.begin(), nb2.end());\n", ""),
    ("critical_without_pushing_cofacets",
     "            make_critical(c);\n            for (int b : ls.cofacets_in_L(c))",
     "            make_critical(c);\n            for (int b : std::vector<int>())"),
    ("dag_keeps_own_partner", "        if (uint32_t(q) == own) continue;\n", ""),
    ("count_assign_not_add", "                cnt[w] = after;", "                cnt[w] = cv;"),
    ("min_arcs_swapped", "out[2 * i] = vertex_min[std::min(vs[0], vs[1])];",
     "out[2 * i] = vertex_min[std::max(vs[0], vs[1])];"),
    ("max_arc_sides_swapped", "d[axis] += side ? 1 : -1;", "d[axis] += side ? -1 : 1;"),
    ("boundary_exit_not_none", "if (!g.inside(nxc, nyc, nzc)) { label = NONE; break; }",
     "if (!g.inside(nxc, nyc, nzc)) { label = uint32_t(c); break; }"),
    ("junction_threshold", "if (dag_out(g, pair_of, c).size() > 1) {", "if (dag_out(g, pair_of, c).size() > 0) {"),
    ("dead_paths_kept", "                if (nxt.empty()) break;  // dead path",
     "                if (nxt.empty()) { mn->m[u_is_saddle ? 3 : 2][{urank, 0}] += 1; break; }"),
    ("arc_walk_repeats_the_vertex", "                res->cells.push_back(uint32_t(g.vertex_cell(w)));\n                v = w;",
     "                res->cells.push_back(uint32_t(g.vertex_cell(v)));\n                v = w;"),
    ("simplify_allows_strangulations", "if (it == adj[size_t(p)].end() || it->second != 1) continue;  // S2",
     "if (it == adj[size_t(p)].end() || it->second < 1) continue;  // S2"),
    ("simplify_reroutes_sum_not_product", "const uint64_t add = a.second * b.second;",
     "const uint64_t add = a.second + b.second;"),
    ("simplify_most_persistent_first", "const Key k = *queue.begin();\n        queue.erase(queue.begin());",
     "const Key k = *std::prev(queue.end());\n        queue.erase(std::prev(queue.end()));"),
    ("rounds_select_one_link_minima", "for (const auto& kv : adj[size_t(u)]) m2[size_t(u)] = std::min(m2[size_t(u)], m1[size_t(kv.first)]);",
     "for (const auto& kv : adj[size_t(u)]) m2[size_t(u)] = std::min(m2[size_t(u)], m0[size_t(kv.first)]);"),
    ("ss_arc_quad_of_the_wrong_cell", "res->cells.push_back(pair_of[next]);  // the quad between e and next",
     "res->cells.push_back(pair_of[e]);  // the quad between e and next"),
    ("packed_codes_x_sides_swapped", "    if (bx == ax - 1) return 1;\n    if (bx == ax + 1) return 2;",
     "    if (bx == ax - 1) return 2;\n    if (bx == ax + 1) return 1;"),
]


def _run_pins():
    """Run a fast subset of the pins; return how many of them failed."""
    checks = []
    for f in pins._fields_small()[:8]:
        checks.append(lambda f=f: pins.test_invariants_and_persistence(f))
    checks += [lambda s=s: pins.test_vertex_pairs_are_steepest_descent(s) for s in range(2)]
    checks += [lambda s=s: pins.test_dstar_matches_vpath_enumeration_and_paper_products(s) for s in (0, 1, 6)]
    checks += [lambda s=s: pins.test_min_labels_are_steepest_descent(s) for s in range(2)]
    checks += [lambda s=s: pins.test_max_labels_properties(s) for s in range(2)]
    checks += [lambda s=s: pins.test_reachable_and_junctions(s) for s in range(2)]
    checks.append(pins.test_cosine_lattice_counts)
    checks += [lambda s=s: pins.test_packed_words_decode_to_the_gradient_pairs(s) for s in range(2)]
    checks += [lambda s=s: pins.test_arc_cells_are_the_v_paths_of_the_arcs(s) for s in range(2)]
    checks += [lambda s=s: pins.test_ss_arc_cells_are_the_single_v_paths(s) for s in (0, 4)]
    checks += [lambda s=s: pins.test_simplification_matches_brute_force_replay(s) for s in range(2)]
    checks += [pins.test_simplification_two_wells_closed_form, pins.test_simplification_cosine_lattice_closed_form]
    checks += [lambda s=s: pins.test_simplification_rounds_match_brute_force_and_the_serial_order(s) for s in range(2)]
    failed = 0
    for c in checks:
        try:
            c()
        except Exception:  # an assertion, or an oracle status error caused by the mutant
            failed += 1
    return failed


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(name, old, new, tmp_path):
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"  # every copy of the line is mutated
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", lib, str(path)])
    with oracle.swap_library(lib):
        failed = _run_pins()
    assert failed > 0, f"no pin rejects the mutant {name}"


def test_unmutated_oracle_passes_the_same_subset():
    assert _run_pins() == 0


def test_prefix_clause_is_immaterial(tmp_path):
    """Reading R2 breaks ties between a key and its proper prefix by calling the prefix
    smaller. Flipping that clause never changes the pairing: exhaustively over all 8!
    vertex orders of one cube, and on random orders of a 3^3 grid (whose centre vertex has
    the full 27-cell star). So the clause is a convention that no output depends on."""
    import numpy as np

    src = open(oracle._SRC).read()
    old = "        return ka.size() < kb.size();"
    assert src.count(old) == 1
    path = tmp_path / "flip.cpp"
    path.write_text(src.replace(old, "        return ka.size() > kb.size();"))
    lib = str(tmp_path / "libflip.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", lib, str(path)])
    import itertools
    fields_ = [np.array(p, dtype=np.float32).reshape(2, 2, 2) for p in itertools.permutations(range(8))]
    rng = np.random.default_rng(0)
    fields_ += [rng.permutation(27).astype(np.float32).reshape(3, 3, 3) for _ in range(3000)]
    base = [oracle.gradient(f) for f in fields_]
    with oracle.swap_library(lib):
        flipped = [oracle.gradient(f) for f in fields_]
    assert all(np.array_equal(a, b) for a, b in zip(base, flipped))
