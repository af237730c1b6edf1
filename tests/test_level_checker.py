"""The Proposition 2 checker used at sizes the oracle cannot reach
(oracle/check_levels.cpp) accepts the oracle's levels and rejects each kind of
wrong level: numbering out of order, two blocks merged, one block split."""
import numpy as np

import oracle
from paper_1210_0748_gb300 import synth


def _canon(ids):
    _, first, inv = np.unique(ids, return_index=True, return_inverse=True)
    rank = np.argsort(np.argsort(first))
    return rank[inv].astype(np.uint32)


def test_checker_accepts_oracle_levels_and_rejects_wrong_ones():
    g = synth.config_single_large(scale=1 / 256, seed=21)
    ref = oracle.kbisim_graph(g, 4, early_stop=False)
    for lev in range(1, 5):
        code, blocks, _ = oracle.check_level(g, ref.pids[lev - 1], ref.pids[lev], threads=4)
        assert code == 0 and blocks == ref.counts[lev], lev
    prev, cur = ref.pids[1], ref.pids[2].copy()
    sizes = np.bincount(cur)
    # numbering out of order: swap ids 0 and 1
    bad = cur.copy()
    bad[cur == 0], bad[cur == 1] = 1, 0
    assert oracle.check_level(g, prev, bad)[0] == 1
    # two blocks merged (renumbered canonically)
    b = int(np.nonzero(sizes >= 1)[0][5])
    merged = cur.copy()
    merged[cur == b] = cur[cur == b + 1][0] if (cur == b + 1).any() else 0
    assert oracle.check_level(g, prev, _canon(merged))[0] == 2
    # one block split (renumbered canonically)
    big = int(np.nonzero(sizes >= 2)[0][0])
    split = cur.astype(np.int64)
    split[np.nonzero(cur == big)[0][-1]] = cur.max() + 1
    assert oracle.check_level(g, prev, _canon(split))[0] == 3
