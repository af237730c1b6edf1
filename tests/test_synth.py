"""Seeded input generators: determinism and the stated shapes."""
import numpy as np

from paper_1210_0748_gb300 import synth


def test_small_config_shape_and_determinism():
    a = synth.config_single_small()
    b = synth.config_single_small()
    assert a.num_nodes == 100_000 and a.num_edges == 1_000_000
    for x, y in ((a.offsets, b.offsets), (a.dst, b.dst), (a.edge_label, b.edge_label),
                 (a.node_label, b.node_label)):
        assert np.array_equal(x, y)
    d = a.degrees()
    assert d.min() >= 1 and d.max() <= 10_000
    assert a.dst.max() < a.num_nodes
    assert set(np.unique(a.edge_label).tolist()) == {0, 1, 2, 3}
    assert set(np.unique(a.node_label).tolist()) == set(range(8))


def test_powerlaw_scaled_shape():
    g = synth.config_single_large(scale=1 / 256)
    assert g.num_nodes == 62_500 and g.num_edges == 1_000_000
    d = g.degrees()
    assert d.sum() == g.num_edges and d.min() >= 1 and d.max() <= 1_000_000
    assert g.edge_label.max() < 32 and g.node_label.max() < 16
    # Zipf labels: label 0 is the most frequent
    assert np.bincount(g.edge_label).argmax() == 0
    # preferential targets: heavy in-degree skew
    indeg = np.bincount(g.dst, minlength=g.num_nodes)
    assert indeg.max() > 50 * indeg.mean()
    other = synth.config_single_large(scale=1 / 256, seed=7)
    assert not np.array_equal(other.dst, g.dst)


def test_from_coo_groups_by_source():
    g = synth.from_coo(4, [3, 0, 3, 1], [0, 1, 2, 3], [5, 6, 7, 8], [0, 0, 1, 1])
    assert g.offsets.tolist() == [0, 1, 2, 2, 4]
    assert g.dst.tolist() == [1, 3, 0, 2] and g.edge_label.tolist() == [6, 8, 5, 7]
    assert g.src().tolist() == [0, 1, 3, 3]


def test_batched_config_shape():
    graphs, ks = synth.config_batched(count=12)
    again, ks2 = synth.config_batched(count=12)
    assert ks == ks2 and all(1 <= k <= 10 for k in ks)
    for g, h in zip(graphs, again):
        assert 1_000 <= g.num_edges <= 1_000_000
        assert g.num_nodes == g.num_edges // 8
        assert int(g.offsets[-1]) == g.num_edges
        assert np.array_equal(g.dst, h.dst)
        assert int(g.node_label.max()) < 8 and int(g.edge_label.max()) < 4
