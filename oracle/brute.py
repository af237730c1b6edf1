"""Brute-force k-bisimilarity straight from Definition 1 (TEST INFRASTRUCTURE).

For tiny graphs only.  B[j][u][v] is True iff u and v are j-bisimilar:

* B[0][u][v]: lambda_N(u) == lambda_N(v)                        (condition 1)
* B[j][u][v]: B[0][u][v], and every out-edge (u, l, u') is matched by an
  out-edge (v, l, v') with B[j-1][u'][v']                        (condition 2)
  and every out-edge of v is matched by one of u the same way    (condition 3)

The relation is then turned into identifiers by ranking its classes by their
smallest node id.  Nothing here uses signatures, sorting or maps, so it
checks the oracle's signature refinement (Proposition 2) independently.
"""
from __future__ import annotations


def relations(num_nodes, node_label, edges, k):
    """edges: iterable of (src, label, dst).  Returns [B_0, ..., B_k]."""
    n = num_nodes
    out = [[] for _ in range(n)]
    for s, l, t in edges:
        out[s].append((l, t))
    b0 = [[node_label[u] == node_label[v] for v in range(n)] for u in range(n)]
    rel = [b0]
    for _ in range(k):
        prev = rel[-1]
        cur = [[False] * n for _ in range(n)]
        for u in range(n):
            for v in range(n):
                if not b0[u][v]:
                    continue
                ok = all(any(lu == lv and prev[tu][tv] for lv, tv in out[v]) for lu, tu in out[u])
                ok = ok and all(any(lv == lu and prev[tv][tu] for lu, tu in out[u])
                                for lv, tv in out[v])
                cur[u][v] = ok
        rel.append(cur)
    return rel


def canonical_ids(rel):
    """Identifiers of an equivalence relation, classes ranked by smallest member."""
    n = len(rel)
    ids = [-1] * n
    nxt = 0
    for u in range(n):
        if ids[u] >= 0:
            continue
        for v in range(u, n):
            if rel[u][v]:
                ids[v] = nxt
        nxt += 1
    return ids


def kbisim_brute(num_nodes, node_label, edges, k):
    """Identifiers for levels 0..k computed from Definition 1 alone."""
    return [canonical_ids(r) for r in relations(num_nodes, node_label, list(edges), k)]
