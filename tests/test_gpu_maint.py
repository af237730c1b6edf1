"""Incremental maintenance (Section 4, Algorithm 3) through kbisim_update:
after every batch the levels equal the oracle's recomputation of the updated
graph (oracle.update.MultiGraph: apply the batch to the edge multiset, then
Algorithm 1), bit for bit, and the update takes the frontier path when the
frontier is small (kbisim_update_info)."""
import numpy as np
import pytest

from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim
from tests import golden_io
from tests.gpu_util import assert_same, graph_from_edges

pytestmark = pytest.mark.gpu


def _mg(g):
    from oracle.update import MultiGraph
    return MultiGraph(g.num_nodes, g.node_label, g.src(), g.dst, g.edge_label)


def _random_batch(rng, mg, n_ins, n_del, n_add=0, labels=3, node_labels=3):
    add = rng.integers(0, node_labels, n_add).astype(np.uint32)
    alive = np.nonzero(np.array(mg.alive + [1] * n_add, bool))[0]
    ins = (rng.choice(alive, n_ins).astype(np.uint32), rng.choice(alive, n_ins).astype(np.uint32),
           rng.integers(0, labels, n_ins).astype(np.uint32))
    s, d, l = mg.coo()
    pick = rng.choice(s.size, min(s.size, n_del), replace=False)
    dels = (s[pick], d[pick], l[pick])
    return add, ins, dels


@pytest.mark.parametrize("early_stop", [True, False])
def test_incremental_updates_equal_the_oracle(early_stop):
    """Small batches of edge inserts, edge deletes (some repeated or absent)
    and node additions on a 5000-node multigraph with out-degree hubs: every
    batch after the first runs on the frontier path."""
    rng = np.random.default_rng(5)
    n = 5000
    g = synth.random_small_graph(n, 12_000, node_labels=3, edge_labels=3, seed=9)
    hub_s = np.full(8000, 11, np.uint32)
    hub_d = rng.integers(0, n, 8000).astype(np.uint32)
    hub_l = rng.integers(0, 3, 8000).astype(np.uint32)
    g = synth.from_coo(n, np.concatenate([g.src(), hub_s]), np.concatenate([g.dst, hub_d]),
                       np.concatenate([g.edge_label, hub_l]), g.node_label)
    mg = _mg(g)
    k = 4
    paths = []
    with KBisim(early_stop=early_stop, maintain="always") as kb:
        kb.build(g, k)
        for step in range(8):
            add, ins, dels = _random_batch(rng, mg, int(rng.integers(1, 12)), int(rng.integers(0, 8)),
                                           n_add=int(step % 3 == 1))
            dl = [np.concatenate([x, x[:1]]) for x in dels]  # one repeated deletion
            want_missing = mg.apply(add, list(zip(*ins)), list(zip(*dl)))
            res, missing = kb.update(k, add_node_label=add, ins=ins, dels=tuple(dl))
            assert missing == want_missing
            assert_same(res, kb.all_pids(k), mg.kbisim(k, early_stop=early_stop))
            paths.append(kb.update_info())
    assert sum(p["incremental"] for p in paths) >= 6, paths
    assert all(p["frontier_nodes"] < n for p in paths if p["incremental"])


def test_in_place_batches_on_a_large_graph():
    """Batches of edge inserts and deletes on the 250K-node power-law graph,
    applied to the edge table in place (every touched node keeps its degree
    class, hubs included), with and without incremental maintenance."""
    rng = np.random.default_rng(12)
    g = synth.config_single_large(scale=1 / 64, seed=6)
    mg = _mg(g)
    k = 3
    with KBisim() as kb, KBisim(maintain=False) as plain:
        kb.build(g, k)
        plain.build(g, k)
        d = np.diff(g.offsets.astype(np.int64))
        hubs = np.nonzero(d > 5000)[0]
        assert hubs.size > 0
        for step in range(4):
            # insertions into distinct nodes of out-degree 10..12 (at most one
            # per batch and four in all, so they stay in class 9..16) and
            # hubs; deletions of hub edges (hubs stay hubs)
            small = np.nonzero((d >= 10) & (d <= 12))[0]
            s_ins = np.concatenate([rng.choice(small, 40, replace=False), rng.choice(hubs, 10)]).astype(np.uint32)
            ins = (s_ins, rng.integers(0, g.num_nodes, 50).astype(np.uint32), rng.integers(0, 32, 50).astype(np.uint32))
            s, dd, l = mg.coo()
            cand_e = np.nonzero(np.isin(s, hubs))[0]
            pick = rng.choice(cand_e, 50, replace=False)
            dels = (s[pick], dd[pick], l[pick])
            mg.apply(ins=list(zip(*ins)), dels=list(zip(*dels)))
            ref = mg.kbisim(k)
            r1, miss = kb.update(k, ins=ins, dels=dels)
            assert miss == 0
            info = kb.update_info()
            assert info["in_place"], info
            r2, _ = plain.update(k, ins=ins, dels=dels)
            assert plain.update_info()["in_place"]
            assert_same(r1, kb.all_pids(k), ref)
            assert_same(r2, plain.all_pids(k), ref)
            d = d + np.bincount(s_ins, minlength=g.num_nodes)


def test_tables_4_and_5_on_the_frontier_path():
    """The paper's Add_Edges examples: Figure 1 plus edge (2, l, 7) with node 7
    added (Table 4), and plus edge (6, l, 5) (Table 5), each as an update of a
    built handle, against the tables as printed."""
    for fix in ("table4_add_edge_2l7.txt", "table5_add_edge_6l5.txt"):
        base = golden_io.load("fig1_table1.txt")
        upd = golden_io.Fixture()
        upd._nlab, upd._elab = base._nlab, base._elab
        upd = golden_io.load(fix, base=upd)
        names = list(base.node_names) + [a for a, _ in upd.add_nodes]
        g = graph_from_edges(len(base.node_names), base.node_label, base.edges)
        ins = [(names.index(a), names.index(b), l) for a, l, b in upd.add_edges]
        with KBisim(early_stop=False, maintain="always") as kb:
            kb.build(g, 2)
            kb.update(2, add_node_label=[l for _, l in upd.add_nodes],
                      ins=tuple(np.array(x, dtype=np.uint32) for x in zip(*ins)))
            assert kb.update_info()["incremental"], kb.update_info()
            for lev in range(3):
                assert kb.pids(lev).tolist() == golden_io.canonical(upd.pids[lev]), (fix, lev)


def test_switch_back_and_recompute_agree():
    """A batch that touches most nodes switches back to the full computation;
    a batch with a node deletion recomputes; maintain=False always recomputes.
    All three give the oracle's levels, and later small batches go back to the
    frontier path."""
    rng = np.random.default_rng(8)
    g = synth.config_single_large(scale=1 / 2048, seed=4)  # 7.8K nodes, 125K edges
    mg = _mg(g)
    k = 3
    with KBisim(maintain="always") as kb, KBisim(maintain=False) as plain:
        kb.build(g, k)
        plain.build(g, k)
        batches = [_random_batch(rng, mg, 4000, 500, labels=32, node_labels=16),
                   _random_batch(rng, mg, 3, 2, labels=32, node_labels=16),
                   _random_batch(rng, mg, 5, 1, labels=32, node_labels=16)]
        for i, (add, ins, dels) in enumerate(batches):
            mg.apply(add, list(zip(*ins)), list(zip(*dels)))
            ref = mg.kbisim(k)
            r1, _ = kb.update(k, ins=ins, dels=dels)
            info = kb.update_info()
            r2, _ = plain.update(k, ins=ins, dels=dels)
            assert plain.update_info()["reason"] == "off"
            assert_same(r1, kb.all_pids(k), ref)
            assert_same(r2, plain.all_pids(k), ref)
            if i == 0:
                assert not info["incremental"] and info["reason"] == "frontier", info
        # a node deletion recomputes, then the next small batch is incremental again
        victim = int(np.nonzero(np.array(mg.alive))[0][3])
        mg.apply(del_nodes=[victim])
        r, _ = kb.update(k, del_nodes=np.array([victim], np.uint32))
        assert kb.update_info()["reason"] == "deletes"
        assert_same(r, kb.all_pids(k), mg.kbisim(k))
        add, ins, dels = _random_batch(rng, mg, 2, 1, labels=32, node_labels=16)
        mg.apply(add, list(zip(*ins)), list(zip(*dels)))
        r, _ = kb.update(k, ins=ins, dels=dels)
        assert kb.update_info()["incremental"]
        assert_same(r, kb.all_pids(k), mg.kbisim(k))


def test_long_signatures_in_the_store():
    """A 12K-edge hub through the signature stores: a new edge gives it a new
    long signature (stored after the lookup pass), a duplicate of one of its
    edges leaves its signature as stored (compared element by element through
    a set in global memory), and deleting the duplicate again too.  Every
    step equals the oracle and runs on the frontier path."""
    rng = np.random.default_rng(21)
    n = 20_000
    hub_t = rng.permutation(n)[:12_000].astype(np.uint32)
    hub_l = rng.integers(0, 3, hub_t.size).astype(np.uint32)
    other = 40_000
    src = np.concatenate([np.zeros(hub_t.size, np.uint32), rng.integers(1, n, other).astype(np.uint32)])
    dst = np.concatenate([hub_t, rng.integers(0, n, other).astype(np.uint32)])
    lab = np.concatenate([hub_l, rng.integers(0, 3, other).astype(np.uint32)])
    nl = rng.integers(0, 2, n).astype(np.uint32)
    g = synth.from_coo(n, src, dst, lab, nl)
    mg = _mg(g)
    k = 3
    dup = (np.array([0], np.uint32), hub_t[:1].copy(), hub_l[:1].copy())
    steps = [dict(ins=(np.array([0], np.uint32), np.array([int(hub_t[5]) ^ 1], np.uint32), np.array([2], np.uint32))),
             dict(ins=dup), dict(dels=dup)]
    with KBisim(maintain="always") as kb:
        kb.build(g, k)
        for st in steps:
            ins, dels = st.get("ins", ()), st.get("dels", ())
            mg.apply(ins=list(zip(*ins)) if len(ins) else [], dels=list(zip(*dels)) if len(dels) else [])
            res, _ = kb.update(k, ins=ins, dels=dels)
            assert kb.update_info()["incremental"], kb.update_info()
            assert_same(res, kb.all_pids(k), mg.kbisim(k))


def test_timed_choice_between_the_paths():
    """maintain=True times both paths on the handle: the first two updates
    take the frontier path (the first, which allocates that path's scratch,
    is not timed), the third recomputes to compare (reason "cost"), and later
    ones take whichever measured cheaper, trying the frontier path again after
    16 recomputations.  Every level equals a handle that always recomputes,
    and the last ones the oracle."""
    rng = np.random.default_rng(31)
    g = synth.config_single_large(scale=1 / 512, seed=8)  # 31K nodes, 500K edges
    mg = _mg(g)
    k = 3
    reasons = []
    with KBisim() as kb, KBisim(maintain=False) as plain:
        kb.build(g, k)
        plain.build(g, k)
        for step in range(24):
            add, ins, dels = _random_batch(rng, mg, 20, 10, labels=32, node_labels=16)
            mg.apply(add, list(zip(*ins)), list(zip(*dels)))
            r1, _ = kb.update(k, ins=ins, dels=dels)
            r2, _ = plain.update(k, ins=ins, dels=dels)
            reasons.append(kb.update_info()["reason"])
            assert list(r1.counts) == list(r2.counts)
            for lev in range(k + 1):
                assert np.array_equal(kb.pids(lev), plain.pids(lev)), (step, lev)
        assert_same(r1, kb.all_pids(k), mg.kbisim(k))
    assert reasons[0] in ("incremental", "frontier") and reasons[1] in ("incremental", "frontier"), reasons
    assert reasons[2] == "cost", reasons
    assert set(reasons) <= {"incremental", "frontier", "cost"}, reasons
    run = 0
    for r in reasons[3:]:  # never more than 15 recomputations in a row on cost
        run = run + 1 if r == "cost" else 0
        assert run <= 15, reasons


def test_frontier_path_on_a_power_law_graph_all_levels():
    """The frontier path on the 250K-node power-law graph (every degree class,
    hubs, targets of in-degree in the thousands), batches of 200 edges: after
    every batch all levels equal those of a handle that recomputes, which the
    other tests tie to the oracle."""
    rng = np.random.default_rng(57)
    g = synth.config_single_large(scale=1 / 64, seed=11)
    mg = _mg(g)
    k = 3
    with KBisim(maintain="always") as kb, KBisim(maintain=False) as plain:
        kb.build(g, k)
        plain.build(g, k)
        inc = 0
        for step in range(6):
            add, ins, dels = _random_batch(rng, mg, 100, 100, labels=32, node_labels=16)
            mg.apply(add, list(zip(*ins)), list(zip(*dels)))
            r1, _ = kb.update(k, ins=ins, dels=dels)
            r2, _ = plain.update(k, ins=ins, dels=dels)
            inc += kb.update_info()["incremental"]
            assert list(r1.counts) == list(r2.counts)
            for lev in range(k + 1):
                assert np.array_equal(kb.pids(lev), plain.pids(lev)), (step, lev)
        assert inc >= 4


def test_store_key_widths():
    """The stores use 32-bit element words when node labels and twice the
    node count fit beside the edge label bits, 64-bit words otherwise: node
    labels up to 2^31 take the 64-bit words; a small graph that gains nodes
    until they no longer fit switches back once and rebuilds its stores.  Every
    batch equals the oracle."""
    rng = np.random.default_rng(61)
    g = synth.random_small_graph(3000, 12_000, node_labels=3, edge_labels=3, seed=3)
    wide = rng.integers(0, 2**31, g.num_nodes).astype(np.uint32)
    g = synth.from_coo(g.num_nodes, g.src(), g.dst, g.edge_label, wide)
    mg = _mg(g)
    with KBisim(maintain="always") as kb:
        kb.build(g, 3)
        for _ in range(4):
            add, ins, dels = _random_batch(rng, mg, 6, 3)
            mg.apply(add, list(zip(*ins)), list(zip(*dels)))
            res, _ = kb.update(3, ins=ins, dels=dels)
            assert_same(res, kb.all_pids(3), mg.kbisim(3))
    small = synth.random_small_graph(50, 150, node_labels=2, edge_labels=2, seed=4)
    mg = _mg(small)
    reasons = []
    with KBisim(maintain="always") as kb:
        kb.build(small, 3)
        for step in range(6):
            add, ins, dels = _random_batch(rng, mg, 4, 2, n_add=30, labels=2, node_labels=2)
            mg.apply(add, list(zip(*ins)), list(zip(*dels)))
            res, _ = kb.update(3, add_node_label=add, ins=ins, dels=dels)
            reasons.append(kb.update_info()["reason"])
            assert_same(res, kb.all_pids(3), mg.kbisim(3))
    assert "capacity" in reasons, reasons


@pytest.mark.parametrize("wide", [False, True])
def test_stores_grow_during_updates(monkeypatch, wide):
    """Stores built with 64 words of room (KBISIM_FAULT_STORE_ROOM) on a graph
    of few blocks take a batch that gives 3000 nodes new signatures: the pool
    and the label arrays grow and the table is rehashed, keeping what they
    hold, and the update stays on the frontier path; a second batch takes
    500 of those nodes back to no out-edges, signatures stored at the build.
    With 32-bit element words (node labels 5/1) and 64-bit ones (node labels
    near 2^31 beside 8-bit edge labels); every batch equals the oracle."""
    monkeypatch.setenv("KBISIM_FAULT_STORE_ROOM", "64")
    rng = np.random.default_rng(71)
    n = 40_000
    nl = np.where(np.arange(n) % 2 == 0, 5, (2**31 - 3) if wide else 1).astype(np.uint32)
    src = np.arange(100, dtype=np.uint32)
    g = synth.from_coo(n, src, src + 1, np.full(100, 255, np.uint32), nl)  # edge labels of 8 bits from the start
    mg = _mg(g)
    k = 3
    srcs = rng.permutation(np.arange(200, n))[:3000].astype(np.uint32)
    a = (np.arange(3000) % 256).astype(np.uint32)
    b = ((np.arange(3000) // 256 + a + 1) % 256).astype(np.uint32)
    first = (np.concatenate([srcs, srcs]), rng.integers(0, n, 6000).astype(np.uint32), np.concatenate([a, b]))
    pick = np.concatenate([np.arange(500), 3000 + np.arange(500)])
    again = tuple(x[pick] for x in first)  # 500 nodes back to no out-edges
    with KBisim(maintain="always") as kb:
        kb.build(g, k)
        for ins, dels in ((first, ()), ((), again)):
            mg.apply(ins=list(zip(*ins)) if ins else [], dels=list(zip(*dels)) if dels else [])
            res, _ = kb.update(k, ins=ins, dels=dels)
            info = kb.update_info()
            assert info["incremental"], info
            assert_same(res, kb.all_pids(k), mg.kbisim(k))


def _update_both(kb, mg, k, ins=(), dels=()):
    """One batch through the handle and the oracle; the handle's levels must
    equal the oracle's and the update must take the frontier path."""
    arr = lambda t: tuple(np.array(x, np.uint32) for x in zip(*t)) if t else ()
    mg.apply(ins=ins, dels=dels)
    res, _ = kb.update(k, ins=arr(ins), dels=arr(dels))
    info = kb.update_info()
    assert info["incremental"], info
    assert_same(res, kb.all_pids(k), mg.kbisim(k))
    return info


def test_unchanged_blocks_keep_their_labels():
    """A block all of whose nodes take one new signature that no label holds
    keeps its label, so nothing propagates to its parents: on a graph whose
    node labels are all distinct (every block a single node) an inserted edge
    leaves the frontier at its source on every level.  A block that moves
    whole keeps its label; a block that splits does not; and a block whose
    old signature another frontier node takes in the same level gets a new
    label.  Every batch equals the oracle."""
    rng = np.random.default_rng(83)
    n, k = 1000, 4
    edges = [(int(a), int(l), int(b)) for a, l, b in zip(rng.integers(0, n, 4000), rng.integers(0, 3, 4000),
                                                       rng.integers(0, n, 4000))]
    g = graph_from_edges(n, np.arange(n, dtype=np.uint32), edges)
    mg = _mg(g)
    with KBisim(maintain="always") as kb:
        kb.build(g, k)
        info = _update_both(kb, mg, k, ins=[(5, 17, 2)])
        assert info["frontier_nodes"] == k, info  # the source alone, on each level
        info = _update_both(kb, mg, k, dels=[(5, 17, 2)])
        assert info["frontier_nodes"] == k, info
    # nodes 0..3 share node label 1, 4 and 5 label 2; 6 is the parent of 0
    # and 1.  Level 1: {0, 1} one block (one edge of label 0 to a label-2
    # node), {2} (label 1), {3} (labels 0 and 1).  Batches as (src, dst, label).
    lab = np.array([1, 1, 1, 1, 2, 2, 3, 4], np.uint32)
    base = [(0, 0, 4), (1, 0, 5), (2, 1, 4), (3, 0, 4), (3, 1, 5), (6, 0, 0), (6, 1, 1), (7, 0, 2)]
    steps = [
        dict(ins=[(0, 4, 2), (1, 5, 2)]),         # {0, 1} moves whole to a signature no label holds
        dict(ins=[(0, 4, 1)]),                    # {0, 1} splits
        dict(ins=[(2, 4, 0)], dels=[(3, 5, 1)]),  # 2 takes {3}'s signature, 3 a signature no label holds
        dict(ins=[(7, 2, 1)], dels=[(2, 4, 1)]),  # 2 takes 3's new one
    ]
    g = graph_from_edges(8, lab, base)
    mg = _mg(g)
    with KBisim(maintain="always") as kb:
        kb.build(g, 3)
        for st in steps:
            _update_both(kb, mg, 3, **st)
    # the hit rule: {x} moves to a new signature while z takes x's old one
    lab = np.array([1, 1, 2, 2], np.uint32)
    g = graph_from_edges(4, lab, [(0, 0, 2), (1, 1, 3)])  # x = 0: (1, {(0, 2)}); z = 1: (1, {(1, 2)})
    mg = _mg(g)
    with KBisim(maintain="always") as kb:
        kb.build(g, 2)
        _update_both(kb, mg, 2, ins=[(0, 2, 3), (1, 3, 0)], dels=[(1, 3, 1)])  # x: new; z: x's old


def test_deletions_on_a_long_hub():
    """Deletions whose source is a hub of 40K edges over 600 distinct triples
    (about 67 copies each, spread over the whole segment): repeated deletions
    of one triple claim distinct copies, deletions beyond a triple's copies
    count as missing, and the levels equal the oracle, on both update paths."""
    rng = np.random.default_rng(97)
    n = 3000
    t = rng.integers(0, 200, 40_000).astype(np.uint32)
    l = rng.integers(0, 3, 40_000).astype(np.uint32)
    other = 9000
    src = np.concatenate([np.full(t.size, 5, np.uint32), rng.integers(0, n, other).astype(np.uint32)])
    dst = np.concatenate([t, rng.integers(0, n, other).astype(np.uint32)])
    lab = np.concatenate([l, rng.integers(0, 3, other).astype(np.uint32)])
    g = synth.from_coo(n, src, dst, lab, rng.integers(0, 3, n).astype(np.uint32))
    for maintain in ("always", False):
        mg = _mg(g)
        with KBisim(maintain=maintain) as kb:
            kb.build(g, 3)
            for step in range(3):
                pick = rng.integers(0, 40_000, 150)
                reps = 1 + (np.arange(pick.size) % 3) * 40  # 1, 41 or 81 deletions of a triple
                ds = np.repeat(np.full(pick.size, 5, np.uint32), reps)
                dt = np.repeat(t[pick], reps)
                dl = np.repeat(l[pick], reps)
                want = mg.apply(dels=list(zip(ds, dt, dl)))
                res, missing = kb.update(3, dels=(ds, dt, dl))
                assert missing == want and want > 0, (missing, want)
                assert_same(res, kb.all_pids(3), mg.kbisim(3))
