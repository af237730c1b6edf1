"""Graph maintenance by apply-then-recompute (TEST INFRASTRUCTURE ONLY).

Section 4 of the paper maintains a k-partition under node insertions
(Algorithm 2), edge insertions (Algorithm 3) and deletions ("Deletions":
an edge delete is handled like an insert; a node delete first removes every
incident edge, then the node).  Its correctness claim (Theorem 2) and its
validation ("Validation of implementations") say the maintained partition is
the one a full rebuild gives.  The oracle therefore applies a batch to the
edge multiset and recomputes from scratch with Algorithm 1, which is correct
by construction.

Batch semantics (the paper assumes new nodes are isolated and new edges join
existing nodes; the remaining choices are this library's):
  1. node additions get ids N, N+1, ... in batch order;
  2. edge insertions add one copy of each (s, l, t) triple;
  3. edge deletions remove one copy of each listed triple, and a triple that
     is not present is ignored (and counted);
  4. node deletions remove every incident edge, then mark the node dead
     (identifier 0xFFFFFFFF at every level, not counted).
"""
from __future__ import annotations

from collections import Counter

import numpy as np

from . import kbisim


class MultiGraph:
    def __init__(self, num_nodes, node_label, src, dst, edge_label):
        self.node_label = [int(x) for x in np.asarray(node_label)]
        self.alive = [1] * int(num_nodes)
        self.edges = Counter()
        for s, t, l in zip(np.asarray(src).tolist(), np.asarray(dst).tolist(),
                           np.asarray(edge_label).tolist()):
            self.edges[(s, l, t)] += 1

    @property
    def num_nodes(self):
        return len(self.node_label)

    def apply(self, add_node_label=(), ins=(), dels=(), del_nodes=()):
        """Apply one batch; ins/dels are iterables of (s, t, l).  Returns the
        number of deletions that named an absent triple."""
        for lab in add_node_label:
            self.node_label.append(int(lab))
            self.alive.append(1)
        n = self.num_nodes
        for s, t, l in ins:
            s, t, l = int(s), int(t), int(l)
            if not (0 <= s < n and 0 <= t < n and self.alive[s] and self.alive[t]):
                raise ValueError("edge insert on a missing or deleted node")
            self.edges[(s, l, t)] += 1
        missing = 0
        for s, t, l in dels:
            key = (int(s), int(l), int(t))
            if self.edges.get(key, 0) > 0:
                self.edges[key] -= 1
                if self.edges[key] == 0:
                    del self.edges[key]
            else:
                missing += 1
        doomed = set()
        for u in del_nodes:
            u = int(u)
            if not (0 <= u < n and self.alive[u]):
                raise ValueError("delete of a missing or deleted node")
            doomed.add(u)
        if doomed:
            for key in [e for e in self.edges if e[0] in doomed or e[2] in doomed]:
                del self.edges[key]
            for u in doomed:
                self.alive[u] = 0
        return missing

    def coo(self):
        src, dst, lab = [], [], []
        for (s, l, t), c in sorted(self.edges.items()):
            src += [s] * c
            dst += [t] * c
            lab += [l] * c
        return (np.array(src, dtype=np.uint32), np.array(dst, dtype=np.uint32),
                np.array(lab, dtype=np.uint32))

    def kbisim(self, k, early_stop=True):
        s, d, l = self.coo()
        return kbisim(self.num_nodes, np.array(self.node_label, dtype=np.uint32), s, d, l, k,
                      early_stop=early_stop, alive=np.array(self.alive, dtype=np.uint8))
