"""The pins catch plausible mistakes in the oracle.

Each case copies the oracle's C++ source, plants one mistake by a textual
edit (a dropped term, a wrong index, a transposed operand, ...), compiles the
copy on the CPU and runs the pin tests against it.  At least one pin must
fail for every planted mistake; the real oracle is untouched.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "kbisim_oracle.cpp")

MUTATIONS = {
    "no_dedupe": ("      s.second.erase(std::unique(s.second.begin(), s.second.end()), s.second.end());\n", ""),
    "child_level0": ("LabelPid(g.lab[e], prev[g.dst[e]])", "LabelPid(g.lab[e], pids[g.dst[e]])"),
    "drop_edge_label": ("LabelPid(g.lab[e], prev[g.dst[e]])", "LabelPid(0, prev[g.dst[e]])"),
    "source_not_target": ("LabelPid(g.lab[e], prev[g.dst[e]])", "LabelPid(g.lab[e], prev[u])"),
    "drop_first_component": ("s.first = first_component ? pids[u] : prev[u];", "s.first = 0;"),
    "in_edges": ("Csr g = group_by_source(n, m, src, dst, edge_label);",
                 "Csr g = group_by_source(n, m, dst, src, edge_label);"),
    "counter_from_one": ("S.insert(std::make_pair(s, (uint32_t)S.size()))",
                         "S.insert(std::make_pair(s, (uint32_t)S.size() + 1))"),
    "stop_vs_level0": ("counts[i] == counts[i - 1]", "counts[i] == counts[0]"),
    "stop_copies_one_short": ("for (uint32_t j = i + 1; j <= k; ++j) {", "for (uint32_t j = i + 2; j <= k; ++j) {"),
    "shared_S_across_levels": ("    std::map<Sig, uint32_t> S;  // fresh signature storage per level\n", ""),
}

PIN_TESTS = [
    pins.test_table1_figure1,
    pins.test_table2_edge_table,
    lambda: pins.test_tables_4_5_updates("table4_add_edge_2l7.txt"),
    lambda: pins.test_tables_4_5_updates("table5_add_edge_6l5.txt"),
    pins.test_table4_duplicate_edge_is_a_set_element,
    pins.test_fig8a_dbest_update_changes_nothing,
    pins.test_fig8b_dworst_update_changes_every_level,
    pins.test_brute_random_small_graphs,
    lambda: pins.test_path_blocks(5),
    lambda: pins.test_invariants_and_full_bisim(1),
    pins.test_empty_and_degenerate,
]


def _mutant(tmp_path, name):
    find, repl = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(find) == 1, "mutation %s no longer applies" % name
    text = text.replace(find, repl)
    if name == "shared_S_across_levels":
        # one S for all levels, declared before the loop
        anchor = "  for (uint32_t i = 1; i <= k; ++i) {\n    std::chrono"
        assert text.count(anchor) == 1
        text = text.replace(anchor, "  std::map<Sig, uint32_t> S;\n" + anchor)
    src = tmp_path / ("m_%s.cpp" % name)
    src.write_text(text)
    lib = tmp_path / ("m_%s.so" % name)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(lib), str(src)])
    return str(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    real = oracle._load()
    mut = ctypes.CDLL(_mutant(tmp_path, name))
    for fn in ("oracle_kbisim", "oracle_full_bisim", "oracle_level0"):
        getattr(mut, fn).argtypes = getattr(real, fn).argtypes
        getattr(mut, fn).restype = getattr(real, fn).restype
    failures = 0
    oracle._lib = mut
    try:
        for t in PIN_TESTS:
            try:
                t()
            except (AssertionError, ValueError, StopIteration):
                failures += 1
    finally:
        oracle._lib = real
    assert failures > 0, "no pin caught mutation %s" % name


def test_delete_pin_catches_deleting_every_copy(monkeypatch):
    """A planted mistake in the update oracle: a deletion that removes every
    copy of its triple instead of one.  The hand-worked delete pin fails."""
    from oracle import update

    def apply_all_copies(self, add_node_label=(), ins=(), dels=(), del_nodes=()):
        missing = 0
        for s, t, l in dels:
            key = (int(s), int(l), int(t))
            if self.edges.pop(key, 0) == 0:
                missing += 1
        return missing

    monkeypatch.setattr(update.MultiGraph, "apply", apply_all_copies)
    with pytest.raises(AssertionError):
        pins.test_delete_removes_one_copy_of_a_repeated_triple()
