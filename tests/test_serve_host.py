"""Request streams of the serving loop (host logic, no GPU)."""
import numpy as np

from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.serve import make_requests


def test_request_stream_shape_and_determinism():
    graphs = [synth.uniform_zipf_graph(m // 10, m, seed=j) for j, m in enumerate([2_000, 10_000, 50_000])]
    a = make_requests(graphs, rate=100.0, count=400, seed=1, batch_min=100, batch_max=20_000)
    b = make_requests(graphs, rate=100.0, count=400, seed=1, batch_min=100, batch_max=20_000)
    assert [(r.t_arrive, r.graph, r.kind, r.k) for r in a] == [(r.t_arrive, r.graph, r.kind, r.k) for r in b]
    t = np.array([r.t_arrive for r in a])
    assert np.all(np.diff(t) >= 0)
    assert 2.5 < t[-1] < 6.0  # about count / rate seconds
    kinds = [r.kind for r in a]
    assert 0.6 < kinds.count("update") / len(kinds) < 0.8
    for r in a:
        g = graphs[r.graph]
        assert 3 <= r.k <= 10
        if r.kind == "update":
            s, d, l = r.ins
            assert s.max() < g.num_nodes and d.max() < g.num_nodes
            ds, dd, dl = r.dels
            # deletions name edges of the generated graph
            for x in range(min(5, ds.size)):
                lo, hi = int(g.offsets[ds[x]]), int(g.offsets[ds[x] + 1])
                assert ((g.dst[lo:hi] == dd[x]) & (g.edge_label[lo:hi] == dl[x])).any()


def test_admission_by_library_enforced_budgets():
    """Idle handles count what they hold, handles with a request in flight
    count their whole budget (the library keeps them within it), and a
    request is admitted only if its own handle's budget fits beside those."""
    from paper_1210_0748_gb300.serve import HbmAdmission, handle_budget
    a = HbmAdmission(total=1000)
    assert a.fits(held_idle=300, budgets_in_flight=400, budget=300)
    assert not a.fits(held_idle=300, budgets_in_flight=400, budget=301)
    assert handle_budget(100) == 400 + (64 << 20)
