"""Pins of the CPU oracle to things other than itself (no GPU needed).

* the paper's worked examples: Table 1 (Figure 1 graph), Table 2, Table 4 and
  Table 5, and the Dbest/Dworst examples of Figure 8;
* brute force from Definition 1 on every graph with up to 3 nodes (edge slots
  none/a/b) and on random graphs with up to 10 nodes;
* closed forms: cycle, path, full b-ary tree, unlabelled graphs at level 1;
* invariants: refinement (Proposition 1), non-decreasing block counts,
  canonical numbering, early stop (Propositions 8-9 in the appendix), the
  stabilised partition equals full bisimulation computed by naive splitting,
  and Definition 3's first component pId_0(u) gives the same partition as
  pId_{i-1}(u).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.update import MultiGraph
from tests import golden_io


def run(n, labels, edges, k, **kw):
    s = np.array([e[0] for e in edges], dtype=np.uint32)
    l = np.array([e[1] for e in edges], dtype=np.uint32)
    d = np.array([e[2] for e in edges], dtype=np.uint32)
    return oracle.kbisim(n, np.array(labels, dtype=np.uint32), s, d, l, k, **kw)


# --- worked examples ---------------------------------------------------------

def test_table1_figure1():
    f = golden_io.load("fig1_table1.txt")
    r = run(len(f.node_names), f.node_label, f.edges, 2, early_stop=False)
    for lev in (0, 1, 2):
        assert r.pids[lev].tolist() == golden_io.canonical(f.pids[lev]), lev
        assert r.counts[lev] == len(set(f.pids[lev]))
    # canonical form written out (paper's counter minus 1, 3 and 7 per level)
    assert r.pids[1].tolist() == [p - 3 for p in f.pids[1]]
    assert r.pids[2].tolist() == [p - 7 for p in f.pids[2]]


def test_table2_edge_table():
    f = golden_io.load("fig1_table1.txt")
    t2 = golden_io.load("table2_et.txt", base=f)
    r = run(len(f.node_names), f.node_label, f.edges, 2, early_stop=False)
    to_canon1 = dict(zip(f.pids[1], golden_io.canonical(f.pids[1])))
    to_canon2 = dict(zip(f.pids[2], golden_io.canonical(f.pids[2])))
    assert r.pids[1].tolist() == [to_canon1[v] for v in t2.nt["old"]]
    assert r.pids[2].tolist() == [to_canon2[v] for v in t2.nt["new"]]
    assert len(t2.et) == len(f.edges)
    for sid, elab, tid, pid_old in t2.et:
        t = f.node(tid)
        assert (f.node(sid), f.elab(elab), t) in f.edges
        assert r.pids[1][t] == to_canon1[pid_old]


def _apply_fixture(base, upd):
    names = list(base.node_names)
    labels = list(base.node_label)
    for name, lab in upd.add_nodes:
        names.append(name)
        labels.append(lab)
    edges = list(base.edges) + [(names.index(a), l, names.index(b)) for a, l, b in upd.add_edges]
    return names, labels, edges


@pytest.mark.parametrize("fix", ["table4_add_edge_2l7.txt", "table5_add_edge_6l5.txt"])
def test_tables_4_5_updates(fix):
    base = golden_io.load("fig1_table1.txt")
    upd = golden_io.Fixture()
    # share label maps with the base graph
    upd._nlab, upd._elab = base._nlab, base._elab
    upd = golden_io.load(fix, base=upd)
    names, labels, edges = _apply_fixture(base, upd)
    r = run(len(names), labels, edges, 2, early_stop=False)
    for lev in (0, 1, 2):
        assert r.pids[lev].tolist() == golden_io.canonical(upd.pids[lev]), (fix, lev)
    # the same through the apply-then-recompute update path
    mg = MultiGraph(len(base.node_names), base.node_label, *base.coo())
    add = [lab for _, lab in upd.add_nodes]
    ins = [(names.index(a), names.index(b), l) for a, l, b in upd.add_edges]
    mg.apply(add_node_label=add, ins=ins)
    r2 = mg.kbisim(2, early_stop=False)
    assert np.array_equal(r2.pids, r.pids)


def test_table4_duplicate_edge_is_a_set_element():
    # Table 4's point: (l, pId(6)) and (l, pId(7)) are one set element.  The
    # same holds for a literal repeated triple.
    f = golden_io.load("fig1_table1.txt")
    edges = list(f.edges) + [f.edges[0], f.edges[3], f.edges[3]]
    r = run(len(f.node_names), f.node_label, edges, 2, early_stop=False)
    for lev in (0, 1, 2):
        assert r.pids[lev].tolist() == golden_io.canonical(f.pids[lev])


def test_fig8a_dbest_update_changes_nothing():
    f = golden_io.load("fig8a_dbest.txt")
    n = len(f.node_names)
    before = run(n, f.node_label, f.edges, 10, early_stop=False)
    names, labels, edges = _apply_fixture(f, f)
    after = run(n, labels, edges, 10, early_stop=False)
    assert np.array_equal(before.pids, after.pids)
    # the root's x edges and the inner nodes' y edges already tell the three
    # depths apart at level 1: {a}, {b, c}, {d, e, f, g}
    assert before.counts.tolist() == [1] + [3] * 10
    assert before.pids[1].tolist() == [0, 1, 1, 2, 2, 2, 2]


def test_fig8b_dworst_update_changes_every_level():
    f = golden_io.load("fig8b_dworst.txt")
    n = len(f.node_names)
    before = run(n, f.node_label, f.edges, 4, early_stop=False)
    assert before.counts.tolist() == [1, 2, 2, 2, 2]
    names, labels, edges = _apply_fixture(f, f)
    after = run(n, labels, edges, 4, early_stop=False)
    # a is split off at level 1 and stays alone; b..e stay together; f alone
    assert after.counts.tolist() == [1, 3, 3, 3, 3]
    for lev in range(1, 5):
        assert after.pids[lev].tolist() == [0, 1, 1, 1, 1, 2]


# --- brute force from Definition 1 -------------------------------------------

def _check_brute(n, labels, edges, k):
    want = brute.kbisim_brute(n, labels, edges, k)
    got = run(n, labels, edges, k, early_stop=False)
    for lev in range(k + 1):
        assert got.pids[lev].tolist() == want[lev], (n, labels, edges, lev)
    got_es = run(n, labels, edges, k, early_stop=True)
    assert np.array_equal(got_es.pids, got.pids)


def test_brute_exhaustive_two_nodes():
    slots = [(u, v) for u in range(2) for v in range(2)]
    for labels in itertools.product(range(2), repeat=2):
        for choice in itertools.product(range(3), repeat=len(slots)):
            edges = [(u, c - 1, v) for (u, v), c in zip(slots, choice) if c]
            _check_brute(2, list(labels), edges, 3)


@pytest.mark.slow
def test_brute_exhaustive_three_nodes():
    # every edge set over 3 nodes with each ordered pair carrying no edge, an
    # 'a' edge or a 'b' edge; node labelings AAA and AAB cover the rest up to
    # renaming of nodes and labels
    slots = [(u, v) for u in range(3) for v in range(3)]
    for labels in ([0, 0, 0], [0, 0, 1]):
        for choice in itertools.product(range(3), repeat=len(slots)):
            edges = [(u, c - 1, v) for (u, v), c in zip(slots, choice) if c]
            _check_brute(3, labels, edges, 3)


def test_brute_random_small_graphs():
    rng = random.Random(1210_0748)
    for _ in range(300):
        n = rng.randint(1, 10)
        m = rng.randint(0, 3 * n)
        nl = rng.randint(1, 3)
        el = rng.randint(1, 3)
        labels = [rng.randrange(nl) for _ in range(n)]
        edges = [(rng.randrange(n), rng.randrange(el), rng.randrange(n)) for _ in range(m)]
        _check_brute(n, labels, edges, rng.randint(0, 6))


def test_brute_multi_labels_on_one_pair():
    # two different labels on the same ordered pair, and repeated triples
    edges = [(0, 0, 1), (0, 1, 1), (0, 0, 1), (2, 0, 1), (3, 1, 1), (3, 0, 1)]
    _check_brute(4, [0, 0, 0, 0], edges, 3)


# --- closed forms --------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 50])
def test_cycle_one_block(n):
    edges = [(u, 0, (u + 1) % n) for u in range(n)]
    r = run(n, [0] * n, edges, 6, early_stop=False)
    assert r.counts.tolist() == [1] * 7


@pytest.mark.parametrize("n", [1, 2, 5, 30])
def test_path_blocks(n):
    edges = [(u, 0, u + 1) for u in range(n - 1)]
    k = 12
    r = run(n, [0] * n, edges, k, early_stop=False)
    assert r.counts.tolist() == [min(j + 1, n) for j in range(k + 1)]
    # level j separates the last j nodes individually
    for j in range(k + 1):
        dist = [n - 1 - u for u in range(n)]
        assert golden_io.canonical([min(d, j) for d in dist]) == r.pids[j].tolist()


@pytest.mark.parametrize("b,h", [(2, 3), (3, 2), (4, 4)])
def test_full_tree_blocks(b, h):
    n = (b ** (h + 1) - 1) // (b - 1)
    edges = [(u, 0, b * u + c + 1) for u in range(n) for c in range(b) if b * u + c + 1 < n]
    k = h + 3
    r = run(n, [0] * n, edges, k, early_stop=False)
    assert r.counts.tolist() == [min(j, h) + 1 for j in range(k + 1)]


def test_unlabelled_random_graph_levels_1_2():
    # one node label and one edge label: level 1 separates sinks from the
    # rest, level 2 has at most 4 blocks (Table 7: Twitter, WikiLinks 2 -> 4)
    rng = np.random.default_rng(5)
    n, m = 400, 900
    s = rng.integers(0, n, m)
    d = rng.integers(0, n, m)
    r = oracle.kbisim(n, np.zeros(n, np.uint32), s, d, np.zeros(m, np.uint32), 3)
    has_out = np.zeros(n, bool)
    has_out[s] = True
    assert has_out.any() and not has_out.all()
    assert r.counts[1] == 2
    assert np.array_equal(r.pids[1] == r.pids[1][np.argmax(has_out)], has_out)
    assert r.counts[2] <= 4


# --- invariants ---------------------------------------------------------------

def _invariants(r, n):
    k = r.pids.shape[0] - 1
    for lev in range(k + 1):
        p = r.pids[lev]
        assert golden_io.canonical(p.tolist()) == p.tolist()
        assert (len(set(p.tolist())) if n else 0) == r.counts[lev]
    for lev in range(1, k + 1):
        assert r.counts[lev] >= r.counts[lev - 1]
        # refinement: each level-lev block lies inside one level-(lev-1) block
        pairs = set(zip(r.pids[lev].tolist(), r.pids[lev - 1].tolist()))
        assert len(pairs) == r.counts[lev]


@pytest.mark.parametrize("seed", range(6))
def test_invariants_and_full_bisim(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 300))
    m = int(rng.integers(0, 4 * n))
    s = rng.integers(0, n, m)
    d = rng.integers(0, n, m)
    el = rng.integers(0, 1 + seed % 3, m)
    nl = rng.integers(0, 1 + seed % 2, n)
    r = oracle.kbisim(n, nl, s, d, el, n + 1, early_stop=False)
    _invariants(r, n)
    # counts stop changing once two consecutive levels agree (appendix,
    # "Partition splitting stop condition")
    c = r.counts.tolist()
    j = next(i for i in range(1, len(c)) if c[i] == c[i - 1])
    assert all(np.array_equal(r.pids[i], r.pids[j]) for i in range(j, len(c)))
    es = oracle.kbisim(n, nl, s, d, el, n + 1, early_stop=True)
    assert es.rounds_run == j
    assert np.array_equal(es.pids, r.pids)
    # the stabilised partition is full bisimulation (appendix, "Connection
    # between localized bisimulation and full bisimulation")
    fb, cnt = oracle.full_bisim(n, nl, s, d, el)
    assert cnt == c[-1]
    assert np.array_equal(fb, r.pids[-1])


@pytest.mark.parametrize("seed", range(4))
def test_definition3_first_component_equivalent(seed):
    rng = np.random.default_rng(100 + seed)
    n = 200
    m = 600
    s, d = rng.integers(0, n, m), rng.integers(0, n, m)
    el, nl = rng.integers(0, 2, m), rng.integers(0, 3, n)
    a = oracle.kbisim(n, nl, s, d, el, 8, early_stop=False, first_component="prev")
    b = oracle.kbisim(n, nl, s, d, el, 8, early_stop=False, first_component="pid0")
    assert np.array_equal(a.pids, b.pids)


def test_empty_and_degenerate():
    r = oracle.kbisim(0, [], [], [], [], 3)
    assert r.counts.tolist() == [0, 0, 0, 0] and r.pids.shape == (4, 0)
    r = oracle.kbisim(5, [3, 3, 1, 3, 1], [], [], [], 0)
    assert r.pids.tolist() == [[0, 0, 1, 0, 1]] and r.rounds_run == 0
    r = oracle.kbisim(5, [3, 3, 1, 3, 1], [], [], [], 4)
    assert r.rounds_run == 1 and r.counts.tolist() == [2, 2, 2, 2, 2]
    with pytest.raises(ValueError):
        oracle.kbisim(2, [0, 0], [0], [2], [0], 1)


def test_update_recompute_with_deletes():
    rng = np.random.default_rng(9)
    n, m = 60, 200
    s, d = rng.integers(0, n, m), rng.integers(0, n, m)
    el, nl = rng.integers(0, 2, m), rng.integers(0, 2, n)
    mg = MultiGraph(n, nl, s, d, el)
    missing = mg.apply(add_node_label=[1, 0], ins=[(60, 3, 1), (2, 61, 0)],
                       dels=[(int(s[0]), int(d[0]), int(el[0])), (0, 0, 7)],
                       del_nodes=[5])
    assert missing == 1
    r = mg.kbisim(6)
    assert r.pids.shape[1] == 62
    assert (r.pids[:, 5] == oracle.DEAD).all()
    alive = np.array(mg.alive, bool)
    for lev in range(r.pids.shape[0]):
        assert r.counts[lev] == len(set(r.pids[lev][alive].tolist()))
    # the same graph built directly, with the dead node's edges gone
    s2, d2, l2 = mg.coo()
    assert not ((s2 == 5) | (d2 == 5)).any()


def _figure1_with_doubled_works_edge():
    """The Figure 1 graph with its edge (1, w, 2) given twice."""
    f = golden_io.load("fig1_table1.txt")
    one, w, two = f.node("1"), f.elab("w"), f.node("2")
    assert (one, w, two) in f.edges
    s, d, l = f.coo(list(f.edges) + [(one, w, two)])
    return f, MultiGraph(len(f.node_names), f.node_label, s, d, l), (one, two, w)


def test_delete_removes_one_copy_of_a_repeated_triple():
    """A deletion removes one stored copy of its triple.  With (1, w, 2) stored
    twice, deleting it once leaves the Figure 1 graph (Table 1 unchanged);
    deleting it twice leaves the graph without that edge, worked by hand from
    Definitions 1-3 (nodes 1..6 as ids 0..5, canonical numbering):
      level 0: M = {1, 2}, P = {3, 4, 5, 6}              -> 0 0 1 1 1 1
      level 1: 1 (M, {l P}); 2 (M, {w M, l P}); 3 and 5 (P, {l M});
               4 (P, {l P}); 6 (P, {})                     -> 0 1 2 3 2 4
      level 2: 3 -> child 1 (block 0), 5 -> child 2 (block 1): split
                                                           -> 0 1 2 3 4 5
    A third deletion names an absent triple and is only counted."""
    f, mg, (one, two, w) = _figure1_with_doubled_works_edge()
    assert mg.apply(dels=[(one, two, w)]) == 0
    r = mg.kbisim(2, early_stop=False)
    for lev in (0, 1, 2):
        assert r.pids[lev].tolist() == golden_io.canonical(f.pids[lev]), lev
    assert mg.apply(dels=[(one, two, w)]) == 0
    r = mg.kbisim(2, early_stop=False)
    assert r.pids[0].tolist() == [0, 0, 1, 1, 1, 1]
    assert r.pids[1].tolist() == [0, 1, 2, 3, 2, 4]
    assert r.pids[2].tolist() == [0, 1, 2, 3, 4, 5]
    assert r.counts.tolist() == [2, 5, 6]
    assert mg.apply(dels=[(one, two, w)]) == 1
    assert mg.kbisim(2, early_stop=False).pids[2].tolist() == [0, 1, 2, 3, 4, 5]
