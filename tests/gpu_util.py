"""Helpers shared by the GPU parity tests: run the CUDA path, run the oracle,
and check full-size results through properties that hold at any size."""
import numpy as np

import oracle
from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim


def gpu_levels(graph, k, **opts):
    """All levels 0..k of ``graph`` (synth.Graph) from the CUDA path."""
    with KBisim(**opts) as kb:
        res = kb.build(graph, k)
        pids = kb.all_pids(k)
    return res, pids


def oracle_levels(graph, k, early_stop=True):
    return oracle.kbisim_graph(graph, k, early_stop=early_stop)


def assert_same(res, pids, ref):
    assert res.counts == ref.counts.tolist(), (res.counts, ref.counts.tolist())
    assert res.rounds_run == ref.rounds_run
    assert pids.shape == ref.pids.shape
    for lev in range(pids.shape[0]):
        if not np.array_equal(pids[lev], ref.pids[lev]):
            bad = np.nonzero(pids[lev] != ref.pids[lev])[0]
            raise AssertionError("level %d differs at %d nodes, first %s: gpu %s oracle %s" % (
                lev, bad.size, bad[:5].tolist(), pids[lev][bad[:5]].tolist(),
                ref.pids[lev][bad[:5]].tolist()))


def graph_from_edges(n, labels, edges):
    src = [e[0] for e in edges]
    lab = [e[1] for e in edges]
    dst = [e[2] for e in edges]
    return synth.from_coo(n, src, dst, lab, labels)


def signature(graph, prev, u):
    """(pId_{i-1}(u), set of (edge label, pId_{i-1}(child))) straight from
    Definition 3, for property checks of large results."""
    lo, hi = int(graph.offsets[u]), int(graph.offsets[u + 1])
    d = graph.dst[lo:hi]
    lab = graph.edge_label[lo:hi].astype(np.uint64)
    elems = np.unique((lab << np.uint64(32)) | prev[d].astype(np.uint64))
    return int(prev[u]), elems.tobytes()


def check_properties(graph, pids, counts, level0_ref, sample=2000, seed=0):
    """Checks that hold at any size:
    * level 0 equals the oracle's level 0;
    * every level is canonical (block r first appears before block r+1), has
      counts[i] blocks and refines the level before (Proposition 1);
    * on a random sample of nodes, pId_i(u) == pId_i(v) iff sig_i(u) ==
      sig_i(v) (Proposition 2), and each sampled node has the signature of
      the first node of its block."""
    rng = np.random.default_rng(seed)
    n = graph.num_nodes
    assert np.array_equal(pids[0], level0_ref)
    for lev in range(pids.shape[0]):
        p = pids[lev]
        assert int(p.max()) + 1 == counts[lev]
        uniq, first = np.unique(p, return_index=True)
        assert uniq.size == counts[lev]
        assert np.all(np.diff(first) > 0), "level %d not canonical" % lev
        if lev:
            assert counts[lev] >= counts[lev - 1]
            pair = (p.astype(np.uint64) << np.uint64(32)) | pids[lev - 1].astype(np.uint64)
            assert np.unique(pair).size == counts[lev], "level %d does not refine" % lev
            nodes = rng.choice(n, size=min(sample, n), replace=False)
            sigs = {}
            for u in nodes.tolist():
                s = signature(graph, pids[lev - 1], u)
                head = int(first[p[u]])
                assert signature(graph, pids[lev - 1], head) == s, (lev, u, head)
                sigs.setdefault(s, set()).add(int(p[u]))
            for s, blocks in sigs.items():
                assert len(blocks) == 1, "equal signatures in different blocks at level %d" % lev
            by_block = {}
            for s, blocks in sigs.items():
                b = next(iter(blocks))
                assert b not in by_block, "one block holds two signatures at level %d" % lev
                by_block[b] = s
