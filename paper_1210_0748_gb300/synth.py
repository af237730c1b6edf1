"""Seeded synthetic graphs shaped like the paper's workloads.

This module only draws random inputs.  It holds none of the k-bisimulation
arithmetic, so the CUDA path and the CPU oracle can both be fed from it
without sharing any of the method's code.

Graphs are directed, node- and edge-labelled multigraphs <N, E, lambda_N,
lambda_E> (Section 2.1 of the paper).  Every generator returns a ``Graph``
whose edges are already grouped by source (CSR): ``offsets[u]..offsets[u+1]``
are the out-edges of node ``u``.  Within a source the edge order is random.

Random numbers come from numpy's PCG64 generator seeded with
``[seed, stream, chunk]`` lists, so a graph is a pure function of its
arguments on any machine.  Per-edge draws are made in chunks on a thread pool.

Workload shapes (the paper's datasets are not available; these stand in for
them, see Table 6 of the paper for the originals):

* ``uniform_zipf_graph``: out-degrees Zipf(s) on [1, dmax] rescaled to exactly
  E, uniform targets, uniform node and edge labels (an RDF-like graph with
  short signatures, like Jamendo/LinkedMDB).
* ``powerlaw_graph``: out-degrees continuous Pareto(alpha) rescaled to exactly
  E with a hub cap, targets drawn with probability proportional to
  (rank+1)^(-1/(alpha-1)) over a seeded permutation of the nodes (a static
  Chung-Lu stand-in for preferential attachment, like Twitter/WikiLinks), Zipf
  node and edge labels.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

DEFAULT_SEED = 0x12100748

# stream ids keep independent draws apart
_S_DEG, _S_TGT, _S_ELAB, _S_NLAB, _S_PERM, _S_BATCH = 1, 2, 3, 4, 5, 6
_CHUNK = 1 << 22


@dataclasses.dataclass
class Graph:
    """A labelled directed multigraph in CSR-by-source form (host arrays)."""

    num_nodes: int
    offsets: np.ndarray      # uint64 [N+1]
    dst: np.ndarray          # uint32 [E]
    edge_label: np.ndarray   # uint8 or uint32 [E]
    node_label: np.ndarray   # uint32 [N]

    @property
    def num_edges(self) -> int:
        return int(self.offsets[-1]) if len(self.offsets) else 0

    def src(self) -> np.ndarray:
        """Source id of every edge (COO view), uint32 [E]."""
        deg = np.diff(self.offsets).astype(np.int64)
        return np.repeat(np.arange(self.num_nodes, dtype=np.uint32), deg)

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def _rng(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed & 0xFFFFFFFFFFFFFFFF, stream, chunk]))


def _rescale_degrees(raw: np.ndarray, total: int, dmin: int, dmax: int) -> np.ndarray:
    """Scale a positive degree sample so that it sums to exactly ``total``.

    Multiply by total/sum, floor, clip to [dmin, dmax], then hand out the
    remaining edges one at a time to the nodes with the largest fractional
    parts (ties to the lower id), skipping nodes at the cap; excess edges (from
    the lower clip) are taken back from the largest degrees.
    """
    n = raw.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    if dmax * n < total or dmin * n > total:
        raise ValueError("degree bounds cannot reach the requested edge count")
    scaled = raw.astype(np.float64) * (total / float(raw.sum()))
    base = np.clip(np.floor(scaled), dmin, dmax).astype(np.int64)
    frac = scaled - np.floor(scaled)
    deficit = total - int(base.sum())
    # stable order: largest fractional part first, lower id on ties
    order = np.lexsort((np.arange(n), -frac))
    while deficit > 0:
        room = order[base[order] < dmax]
        take = room[:deficit]
        base[take] += 1
        deficit -= take.shape[0]
    while deficit < 0:
        order_big = np.lexsort((np.arange(n), -base))
        room = order_big[base[order_big] > dmin]
        take = room[: -deficit]
        base[take] -= 1
        deficit += take.shape[0]
    return base


def _zipf_cdf(num: int, s: float) -> np.ndarray:
    w = np.arange(1, num + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _draw_categorical(cdf: np.ndarray, count: int, seed: int, stream: int,
                      pool: ThreadPoolExecutor, dtype) -> np.ndarray:
    out = np.empty(count, dtype=dtype)

    def work(ci: int) -> None:
        lo = ci * _CHUNK
        hi = min(count, lo + _CHUNK)
        u = _rng(seed, stream, ci).random(hi - lo)
        idx = np.searchsorted(cdf, u, side="right")
        np.minimum(idx, cdf.shape[0] - 1, out=idx)
        out[lo:hi] = idx.astype(dtype)

    list(pool.map(work, range((count + _CHUNK - 1) // _CHUNK)))
    return out


def _pool() -> ThreadPoolExecutor:
    return ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))


def uniform_zipf_graph(num_nodes: int, num_edges: int, *, zipf_s: float = 2.0,
                       dmax: int = 10_000, node_labels: int = 8, edge_labels: int = 4,
                       seed: int = DEFAULT_SEED) -> Graph:
    """Out-degree Zipf(s) on [1, dmax] rescaled to exactly ``num_edges``;
    uniform targets; uniform node labels over ``node_labels`` and edge labels
    over ``edge_labels``."""
    n, m = int(num_nodes), int(num_edges)
    with _pool() as pool:
        if n == 0:
            deg = np.zeros(0, dtype=np.int64)
        else:
            cdf = _zipf_cdf(dmax, zipf_s)
            raw = _draw_categorical(cdf, n, seed, _S_DEG, pool, np.int64) + 1
            deg = _rescale_degrees(raw, m, 1 if m >= n else 0, min(dmax, max(m, 1)))
        offsets = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(deg, out=offsets[1:])
        dst = np.empty(m, dtype=np.uint32)

        def tgt(ci: int) -> None:
            lo = ci * _CHUNK
            hi = min(m, lo + _CHUNK)
            dst[lo:hi] = _rng(seed, _S_TGT, ci).integers(0, n, hi - lo, dtype=np.uint32)

        list(pool.map(tgt, range((m + _CHUNK - 1) // _CHUNK)))
        elab = _draw_categorical(np.arange(1, edge_labels + 1) / edge_labels, m, seed,
                                 _S_ELAB, pool, np.uint8 if edge_labels <= 256 else np.uint32)
        nlab = _draw_categorical(np.arange(1, node_labels + 1) / node_labels, n, seed,
                                 _S_NLAB, pool, np.uint32)
    return Graph(n, offsets, dst, elab, nlab)


def powerlaw_graph(num_nodes: int, num_edges: int, *, alpha: float = 2.1,
                   hub_cap: int = 1_000_000, node_labels: int = 16, node_zipf: float = 1.2,
                   edge_labels: int = 32, edge_zipf: float = 1.5,
                   seed: int = DEFAULT_SEED) -> Graph:
    """Power-law out-degrees and preferential-attachment-like in-degrees.

    Out-degrees: continuous Pareto with pdf ~ x^-alpha on [1, inf), rescaled to
    exactly ``num_edges`` and capped at ``hub_cap``.  Targets: node
    ``perm[r]`` where r has probability ~ (r+1)^(-1/(alpha-1)), drawn by
    inverting the continuous approximation of that distribution.  Labels:
    Zipf over ``node_labels`` / ``edge_labels`` with the given exponents.
    """
    n, m = int(num_nodes), int(num_edges)
    with _pool() as pool:
        raw = np.empty(n, dtype=np.float64)

        def degw(ci: int) -> None:
            lo = ci * _CHUNK
            hi = min(n, lo + _CHUNK)
            u = _rng(seed, _S_DEG, ci).random(hi - lo)
            raw[lo:hi] = np.maximum(1.0, np.rint((1.0 - u) ** (-1.0 / (alpha - 1.0))))

        list(pool.map(degw, range((n + _CHUNK - 1) // _CHUNK)))
        cap = max(1, min(hub_cap, m))
        deg = _rescale_degrees(raw, m, 1 if m >= n else 0, cap) if n else np.zeros(0, np.int64)
        offsets = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(deg, out=offsets[1:])

        perm = _rng(seed, _S_PERM).permutation(n).astype(np.uint32) if n else np.zeros(0, np.uint32)
        beta = 1.0 / (alpha - 1.0)
        gexp = 1.0 - beta
        top = (n + 1.0) ** gexp - 1.0 if abs(gexp) > 1e-12 else np.log(n + 1.0)
        dst = np.empty(m, dtype=np.uint32)

        def tgt(ci: int) -> None:
            lo = ci * _CHUNK
            hi = min(m, lo + _CHUNK)
            u = _rng(seed, _S_TGT, ci).random(hi - lo)
            if abs(gexp) > 1e-12:
                r = (1.0 + u * top) ** (1.0 / gexp) - 1.0
            else:
                r = np.exp(u * top) - 1.0
            ri = np.clip(r.astype(np.int64), 0, n - 1)
            dst[lo:hi] = perm[ri]

        list(pool.map(tgt, range((m + _CHUNK - 1) // _CHUNK)))
        elab = _draw_categorical(_zipf_cdf(edge_labels, edge_zipf), m, seed, _S_ELAB, pool,
                                 np.uint8 if edge_labels <= 256 else np.uint32)
        nlab = _draw_categorical(_zipf_cdf(node_labels, node_zipf), n, seed, _S_NLAB, pool,
                                 np.uint32)
    return Graph(n, offsets, dst, elab, nlab)


def random_small_graph(num_nodes: int, num_edges: int, *, node_labels: int = 2,
                       edge_labels: int = 2, seed: int = 0) -> Graph:
    """Uniform random multigraph (any source, any target, self-loops allowed)
    for small tests; sources are drawn uniformly, then grouped."""
    n, m = int(num_nodes), int(num_edges)
    g = _rng(seed, 99)
    if n == 0:
        m = 0
    src = g.integers(0, max(n, 1), m, dtype=np.uint32)
    dst = g.integers(0, max(n, 1), m, dtype=np.uint32)
    elab = g.integers(0, edge_labels, m, dtype=np.uint32)
    nlab = g.integers(0, node_labels, n, dtype=np.uint32)
    return from_coo(n, src, dst, elab, nlab)


def from_coo(num_nodes: int, src, dst, edge_label, node_label) -> Graph:
    """Group a COO edge list by source (stable) into a ``Graph``."""
    n = int(num_nodes)
    src = np.asarray(src, dtype=np.uint32)
    dst = np.asarray(dst, dtype=np.uint32)
    elab = np.asarray(edge_label, dtype=np.uint32)
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src, minlength=n).astype(np.uint64) if src.size else np.zeros(n, np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    return Graph(n, offsets, dst[order], elab[order], np.asarray(node_label, dtype=np.uint32))


# Named workloads (sizes from the benchmark configurations) --------------------

def config_single_small(seed: int = DEFAULT_SEED + 1) -> Graph:
    """100K nodes, 1M edges, Zipf(2.0) out-degrees capped at 10K, uniform
    targets, 8 node labels and 4 edge labels uniform (k = 5 workload)."""
    return uniform_zipf_graph(100_000, 1_000_000, zipf_s=2.0, dmax=10_000,
                              node_labels=8, edge_labels=4, seed=seed)


def config_single_large(seed: int = DEFAULT_SEED + 2, scale: float = 1.0) -> Graph:
    """16M nodes, 256M edges (times ``scale``), power-law alpha = 2.1 out-degrees,
    preferential-attachment targets, 16 node labels Zipf(1.2), 32 edge labels
    Zipf(1.5) (k = 10 with early stop)."""
    n = max(1, int(round(16_000_000 * scale)))
    m = max(1, int(round(256_000_000 * scale)))
    return powerlaw_graph(n, m, alpha=2.1, hub_cap=1_000_000, node_labels=16, node_zipf=1.2,
                          edge_labels=32, edge_zipf=1.5, seed=seed)


def config_batched(seed: int = DEFAULT_SEED + 3, count: int = 4096):
    """``count`` independent graphs: edge counts log-uniform in [1K, 1M], nodes =
    edges / 8, out-degrees Zipf(2.0) capped at 10K, uniform targets, 8 node
    labels and 4 edge labels uniform (the 100K/1M generator's distributions),
    k uniform in 1..10.  Graph j is drawn with its own seed.  Returns
    (graphs, ks)."""
    rng = _rng(seed, _S_BATCH, 0)
    edges = np.exp(rng.uniform(np.log(1e3), np.log(1e6), count)).astype(np.int64)
    ks = rng.integers(1, 11, count).astype(np.int64)
    graphs = [uniform_zipf_graph(int(e // 8), int(e), zipf_s=2.0, dmax=10_000, node_labels=8, edge_labels=4,
                                 seed=seed * 65_536 + j) for j, e in enumerate(edges.tolist())]
    return graphs, [int(k) for k in ks]


def config_large_single(seed: int = DEFAULT_SEED + 5, scale: float = 1.0) -> Graph:
    """256M nodes, 2B edges (times ``scale``), power-law alpha = 2.0 out-degrees
    with hubs to 1M, preferential-attachment targets, 64 node labels and 16
    edge labels Zipf(1.3) (k = 10)."""
    n = max(1, int(round(256_000_000 * scale)))
    m = max(1, int(round(2_000_000_000 * scale)))
    return powerlaw_graph(n, m, alpha=2.0, hub_cap=1_000_000, node_labels=64, node_zipf=1.3,
                          edge_labels=16, edge_zipf=1.3, seed=seed)


def config_serving(seed: int = DEFAULT_SEED + 4, count: int = 64, scale: float = 1.0):
    """``count`` resident graphs: edge counts log-uniform in [1M, 64M] (times
    ``scale``), nodes = edges / 10, the 100K/1M generator's distributions, and
    an initial k uniform in 3..10.  Returns (graphs, ks)."""
    rng = _rng(seed, _S_BATCH, 1)
    edges = (np.exp(rng.uniform(np.log(1e6), np.log(64e6), count)) * scale).astype(np.int64)
    ks = rng.integers(3, 11, count).astype(np.int64)
    graphs = [uniform_zipf_graph(max(1, int(e // 10)), max(1, int(e)), zipf_s=2.0, dmax=10_000, node_labels=8,
                                 edge_labels=4, seed=seed * 65_536 + j) for j, e in enumerate(edges.tolist())]
    return graphs, [int(k) for k in ks]
