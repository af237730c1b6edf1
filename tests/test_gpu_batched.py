"""Batched build (kbisim_build_many): every graph of a batch gets exactly the
levels, counts and rounds it gets when built alone, and those equal the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim, KBisimError, ERR_INVALID_ARG, ERR_STATE, concat_graphs

pytestmark = pytest.mark.gpu


def _mixed_batch(seed, count):
    """Graphs of uneven sizes, including an empty graph, a single node and a
    graph without edges."""
    rng = np.random.default_rng(seed)
    graphs = [synth.random_small_graph(0, 0, seed=seed), synth.random_small_graph(1, 0, seed=seed + 1),
              synth.random_small_graph(7, 0, node_labels=3, seed=seed + 2)]
    for j in range(count):
        n = int(rng.integers(2, 60))
        m = int(rng.integers(0, 4 * n))
        graphs.append(synth.random_small_graph(n, m, node_labels=int(rng.integers(1, 4)),
                                               edge_labels=int(rng.integers(1, 3)), seed=seed * 1000 + j))
    rng.shuffle(graphs)
    ks = [int(x) for x in rng.integers(0, 7, size=len(graphs))]
    return graphs, ks


def _check_batch(kb, graphs, ks, early_stop=True):
    for j, (g, k) in enumerate(zip(graphs, ks)):
        ref = oracle.kbisim_graph(g, k, early_stop=early_stop)
        rounds, counts = kb.many_info(j)
        assert rounds == ref.rounds_run, (j, rounds, ref.rounds_run)
        assert counts.tolist() == ref.counts.tolist(), (j, counts.tolist(), ref.counts.tolist())
        for lev in range(k + 1):
            got = kb.many_pids(j, lev)
            assert np.array_equal(got, ref.pids[lev]), (j, lev)


@pytest.mark.parametrize("seed", [3, 4])
def test_batch_equals_oracle_per_graph(seed):
    graphs, ks = _mixed_batch(seed, 40)
    with KBisim() as kb:
        kb.build_many(graphs, ks)
        _check_batch(kb, graphs, ks)


def test_batch_without_early_stop():
    graphs, ks = _mixed_batch(9, 20)
    with KBisim(early_stop=False) as kb:
        kb.build_many(graphs, ks)
        _check_batch(kb, graphs, ks, early_stop=False)


def test_batch_equals_solo_builds_with_hubs():
    """Power-law graphs with hubs (every degree class) batched and alone."""
    graphs = [synth.config_single_large(seed=11 + j, scale=s) for j, s in enumerate([1 / 512, 1 / 1024, 1 / 256])]
    graphs.append(synth.uniform_zipf_graph(20_000, 200_000, seed=5))
    ks = [4, 10, 2, 6]
    with KBisim() as kb:
        kb.build_many(graphs, ks)
        for j, (g, k) in enumerate(zip(graphs, ks)):
            with KBisim() as solo:
                res = solo.build(g, k)
                rounds, counts = kb.many_info(j)
                assert rounds == res.rounds_run
                assert counts.tolist() == list(res.counts)
                for lev in range(k + 1):
                    assert np.array_equal(kb.many_pids(j, lev), solo.pids(lev)), (j, lev)


def test_identical_graphs_in_one_batch():
    """Copies of one graph: union blocks span graphs, per-graph ids must not."""
    g = synth.random_small_graph(40, 120, node_labels=2, edge_labels=2, seed=21)
    graphs = [g, g, g]
    with KBisim() as kb:
        kb.build_many(graphs, [5, 5, 5])
        ref = oracle.kbisim_graph(g, 5)
        for j in range(3):
            for lev in range(6):
                assert np.array_equal(kb.many_pids(j, lev), ref.pids[lev])


def test_batch_rejects_bad_input():
    a = synth.random_small_graph(10, 30, seed=1)
    b = synth.random_small_graph(10, 30, seed=2)
    union, starts = concat_graphs([a, b])
    with KBisim() as kb:
        with pytest.raises(KBisimError) as e:
            kb.many_info(0)
        assert e.value.code == ERR_STATE
        bad = synth.Graph(union.num_nodes, union.offsets.copy(), union.dst.copy(), union.edge_label.copy(),
                          union.node_label.copy())
        bad.dst[0] = 15  # an edge of graph 0 into graph 1
        with pytest.raises(KBisimError) as e:
            kb.build_many(None, [3, 3], union=(bad, starts))
        assert e.value.code == ERR_INVALID_ARG
        with pytest.raises(KBisimError) as e:
            kb.build_many(None, [3, 3], union=(union, np.array([0, 12, 20], dtype=np.uint64)[[0, 2, 1]]))
        assert e.value.code == ERR_INVALID_ARG
        kb.build_many([a, b], [2, 3])
        with pytest.raises(KBisimError) as e:
            kb.many_pids(0, 3)  # above k of graph 0
        assert e.value.code == ERR_INVALID_ARG
