"""Serving loop: build and update requests on device-resident graphs.

Each resident graph lives in its own library handle with its own CUDA stream
and its own HBM budget, which the library enforces (kbisim_set_hbm_budget: a
call that would hold more fails with KBISIM_ERR_BUDGET instead of
allocating).  Requests arrive over time (``Request.t_arrive``, seconds from
the start); the loop admits a request as soon as

* its graph has no request in flight (requests on one graph run in arrival
  order, so each result is the one the same sequence gives one at a time),
* a slot is free (at most ``slots`` requests in flight), and
* the server's HBM budget holds the bytes the idle handles hold now, plus the
  budgets of the handles with a request in flight (each may grow up to its
  budget, never past it), plus the budget of the request's own handle,

and runs it on a worker thread (the library call releases the interpreter
lock), so requests on different graphs overlap on the device.  A request
arriving while others run is admitted the moment a slot and memory free up,
not at the end of a batch.

Request kinds: ``update`` (a maintenance batch, then levels 0..k of the
updated graph, Section 4) and ``rebuild`` (levels 0..k from scratch,
Algorithm 1).  Each result records the block counts and a digest of the
level-k identifiers.

Handles recompute on update by default (``maintain=False``): a stream that
spreads its updates over many graphs at varying k gives each handle few
updates in a row, so the signature stores of the frontier path (built once
per graph and k, about one signature pass per level) would rarely pay off;
``Server(maintain=True)`` turns the timed choice of the library on.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import hashlib
import threading
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from .kbisim import ERR_BUDGET, KBisim, KBisimError


@dataclasses.dataclass
class Request:
    rid: int
    t_arrive: float
    graph: int
    kind: str                      # "update" or "rebuild"
    k: int
    ins: Optional[tuple] = None    # (src, dst, label) arrays
    dels: Optional[tuple] = None


@dataclasses.dataclass
class Outcome:
    rid: int
    graph: int
    kind: str
    t_arrive: float
    t_start: float
    t_end: float
    rounds_run: int
    counts: List[int]
    digest: str
    edges: int
    error: str = ""                # "budget": the handle's HBM budget refused the request

    @property
    def latency(self) -> float:
        return self.t_end - self.t_arrive


def _digest(pids: np.ndarray) -> str:
    return hashlib.sha256(pids.tobytes()).hexdigest()[:16]


class HbmAdmission:
    """Admission by HBM budget (host logic).  Every handle h has a budget
    B_h that the library enforces, so a handle with a request in flight never
    holds more than B_h and an idle one holds what it holds now (H_h).  A
    request on handle r is admitted iff
        sum(H_h, h idle) + sum(B_h, h in flight) + B_r <= total,
    so the device never holds more than `total` for the handles."""

    def __init__(self, total: int):
        self.total = int(total)

    def fits(self, held_idle: int, budgets_in_flight: int, budget: int) -> bool:
        return held_idle + budgets_in_flight + budget <= self.total


def handle_budget(held_after_build: int) -> int:
    """Budget of a resident graph's handle: room for an update's second edge
    table and the signature stores of incremental maintenance beside what the
    handle holds after its build."""
    return 4 * int(held_after_build) + (64 << 20)


class Server:
    """Resident graphs (``synth.Graph`` list) with an initial k each."""

    def __init__(self, graphs: Sequence, ks: Sequence[int], *, slots: int = 4, device: int = 0,
                 hbm_budget: Optional[int] = None, maintain=False):
        import torch
        self.torch = torch
        self.device = device
        self.slots = max(1, int(slots))
        self.handles: List[KBisim] = []
        self.budgets: List[int] = []
        self.k = list(int(x) for x in ks)
        for g, k in zip(graphs, self.k):
            stream = torch.cuda.Stream(device=device)
            h = KBisim(device=device, stream=stream, maintain=maintain)
            h.build(g, k)
            b = handle_budget(h.device_bytes)
            h.set_hbm_budget(b)
            self.handles.append(h)
            self.budgets.append(b)
        torch.cuda.synchronize(device)
        free, _ = torch.cuda.mem_get_info(device)
        held = sum(h.device_bytes for h in self.handles)
        self.admission = HbmAdmission(int(hbm_budget) if hbm_budget is not None else held + int(free * 0.8))

    def close(self):
        for h in self.handles:
            h.close()
        self.handles = []

    # -- one request (worker thread) -------------------------------------------
    def _run(self, req: Request, t0: float) -> Outcome:
        h = self.handles[req.graph]
        t_start = time.perf_counter() - t0
        try:
            if req.kind == "update":
                res, _ = h.update(req.k, ins=req.ins if req.ins is not None else (),
                                  dels=req.dels if req.dels is not None else ())
            else:
                res = h.refine(req.k)
            pids = h.pids(req.k)
        except KBisimError as e:
            if e.code != ERR_BUDGET:
                raise
            t_end = time.perf_counter() - t0
            return Outcome(req.rid, req.graph, req.kind, req.t_arrive, t_start, t_end, 0, [], "", h.num_edges,
                           error="budget")
        t_end = time.perf_counter() - t0
        return Outcome(req.rid, req.graph, req.kind, req.t_arrive, t_start, t_end, res.rounds_run,
                       list(res.counts), _digest(pids), h.num_edges)

    # -- the loop ----------------------------------------------------------------
    def serve(self, requests: Sequence[Request], realtime: bool = True) -> List[Outcome]:
        """Run ``requests`` (sorted by arrival).  With realtime, a request is not
        admitted before its arrival time; without, all have arrived at t = 0."""
        reqs = sorted(requests, key=lambda r: (r.t_arrive, r.rid))
        pending: List[Request] = []
        busy: Dict[int, bool] = {}
        inflight: Dict[cf.Future, Request] = {}
        done: List[Outcome] = []
        nxt = 0
        t0 = time.perf_counter()
        lock = threading.Lock()
        with cf.ThreadPoolExecutor(max_workers=self.slots) as pool:
            while nxt < len(reqs) or pending or inflight:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and (not realtime or reqs[nxt].t_arrive <= now):
                    pending.append(reqs[nxt])
                    nxt += 1
                # admit in arrival order; a request waits only for its own graph,
                # a slot and memory
                kept = []
                for r in pending:
                    if len(inflight) < self.slots and not busy.get(r.graph):
                        flying = {x.graph for x in inflight.values()}
                        held_idle = sum(h.device_bytes for i, h in enumerate(self.handles) if i not in flying)
                        in_flight = sum(self.budgets[i] for i in flying)
                        if self.admission.fits(held_idle - self.handles[r.graph].device_bytes, in_flight,
                                               self.budgets[r.graph]) or not inflight:
                            busy[r.graph] = True
                            inflight[pool.submit(self._run, r, t0)] = r
                            continue
                    kept.append(r)
                pending = kept
                timeout = None
                if nxt < len(reqs) and realtime:
                    timeout = max(0.0, reqs[nxt].t_arrive - (time.perf_counter() - t0))
                if inflight:
                    fin, _ = cf.wait(list(inflight), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                    for f in fin:
                        r = inflight.pop(f)
                        busy[r.graph] = False
                        with lock:
                            done.append(f.result())
                elif timeout:
                    time.sleep(timeout)
        return sorted(done, key=lambda o: o.rid)


def make_requests(graphs, rate: float, count: int, seed: int = 0, *, update_frac: float = 0.7,
                  batch_min: int = 1_000, batch_max: int = 1_000_000, k_range=(3, 10)) -> List[Request]:
    """Poisson arrivals at ``rate`` per second; each request targets a graph
    uniformly; ``update_frac`` of them are updates with a batch size
    log-uniform in [batch_min, batch_max] (capped at the graph's edges), half
    insertions of random (src, dst, label) with existing labels and half
    deletions of edges drawn from the graph as generated; the rest are
    rebuilds with k uniform in k_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        gi = int(rng.integers(0, len(graphs)))
        g = graphs[gi]
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        if rng.random() < update_frac and g.num_nodes:
            b = int(np.exp(rng.uniform(np.log(batch_min), np.log(batch_max))))
            b = max(2, min(b, max(2, g.num_edges)))
            ni, nd = b // 2, b - b // 2
            labs = np.unique(g.edge_label) if g.num_edges else np.zeros(1, np.uint32)
            ins = (rng.integers(0, g.num_nodes, ni).astype(np.uint32),
                   rng.integers(0, g.num_nodes, ni).astype(np.uint32),
                   labs[rng.integers(0, labs.size, ni)].astype(np.uint32))
            if g.num_edges:
                e = rng.integers(0, g.num_edges, nd)
                src = (np.searchsorted(g.offsets, e, side="right") - 1).astype(np.uint32)
                dels = (src, g.dst[e].astype(np.uint32), g.edge_label[e].astype(np.uint32))
            else:
                dels = None
            out.append(Request(rid, t, gi, "update", k, ins, dels))
        else:
            out.append(Request(rid, t, gi, "rebuild", k))
    return out


def run_alone(graphs, ks, requests: Sequence[Request], device: int = 0) -> List[Outcome]:
    """The same requests one at a time, in arrival order, on fresh handles."""
    srv = Server(graphs, ks, slots=1, device=device)
    try:
        return srv.serve(requests, realtime=False)
    finally:
        srv.close()
