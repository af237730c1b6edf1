"""CPU oracle for k-bisimulation (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_1210_0748_gb300``) never imports it, and the two
share no code: the oracle is Algorithm 1 of the paper written out with
ordered maps (``kbisim_oracle.cpp``), a brute force from Definition 1
(``brute.py``) and an apply-then-recompute update (``update.py``).

Functions here take plain numpy arrays (COO edges) and return numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbisim_oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "check_levels.cpp")]
_LIB = os.path.join(_HERE, "libkbisim_oracle.so")
_lock = threading.Lock()
_lib = None

DEAD = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host C++ compiler."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            U64 = ctypes.c_uint64
            lib.oracle_kbisim.argtypes = [U64, P, P, U64, P, P, P, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_int, P, P, P, P]
            lib.oracle_kbisim.restype = ctypes.c_int
            lib.oracle_full_bisim.argtypes = [U64, P, U64, P, P, P, P, P]
            lib.oracle_full_bisim.restype = ctypes.c_int
            lib.oracle_level0.argtypes = [U64, P, P, P]
            lib.oracle_level0.restype = U64
            lib.oracle_check_level.argtypes = [U64, P, P, P, ctypes.c_int, P, P, ctypes.c_int, P, P]
            lib.oracle_check_level.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


class Result:
    """pids[i] = pId_i as uint32 [N]; counts[i] = number of blocks of level i."""

    def __init__(self, pids, counts, rounds_run, round_seconds):
        self.pids = pids
        self.counts = counts
        self.rounds_run = rounds_run
        self.round_seconds = round_seconds


def kbisim(num_nodes, node_label, src, dst, edge_label, k, *, early_stop=True,
           first_component="prev", alive=None) -> Result:
    """Algorithm 1 (Build_Bisim): pId_0..pId_k with canonical numbering.

    first_component: "prev" uses pId_{i-1}(u) as the first signature
    component, "pid0" uses pId_0(u) as Definition 3 prints it.
    """
    lib = _load()
    n = int(num_nodes)
    nl, s, d, l = _u32(node_label), _u32(src), _u32(dst), _u32(edge_label)
    m = s.size
    if not (d.size == m and l.size == m and nl.size == n):
        raise ValueError("array sizes disagree")
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, dtype=np.uint8))
    pids = np.zeros((k + 1, max(n, 1)), dtype=np.uint32)[:, :n].copy()
    counts = np.zeros(k + 1, dtype=np.uint64)
    rr = np.zeros(1, dtype=np.uint32)
    secs = np.zeros(max(k, 1), dtype=np.float64)
    rc = lib.oracle_kbisim(n, _ptr(nl), _ptr(al), m, _ptr(s), _ptr(d), _ptr(l), int(k),
                           1 if early_stop else 0, 1 if first_component == "pid0" else 0,
                           _ptr(pids) if pids.size else None, counts.ctypes.data_as(ctypes.c_void_p),
                           rr.ctypes.data_as(ctypes.c_void_p), secs.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("oracle rejected the input (node id out of range or edge on a dead node)")
    return Result(pids, counts.astype(np.int64), int(rr[0]), secs[: int(rr[0])])


def kbisim_graph(g, k, **kw) -> Result:
    """``kbisim`` on a ``synth.Graph`` (CSR) instance."""
    return kbisim(g.num_nodes, g.node_label, g.src(), g.dst, g.edge_label, k, **kw)


def full_bisim(num_nodes, node_label, src, dst, edge_label):
    """Full bisimulation partition by naive splitting; returns (ids, count)."""
    lib = _load()
    n = int(num_nodes)
    nl, s, d, l = _u32(node_label), _u32(src), _u32(dst), _u32(edge_label)
    out = np.zeros(n, dtype=np.uint32)
    cnt = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_full_bisim(n, _ptr(nl), s.size, _ptr(s), _ptr(d), _ptr(l), _ptr(out),
                               cnt.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return out, int(cnt[0])


def check_level(g, prev, cur, threads=None):
    """Check candidate level ``cur`` of CSR graph ``g`` (a ``synth.Graph``)
    against the previous level ``prev`` through Proposition 2 (check_levels.cpp):
    returns (code, blocks, bad_node); code 0 means cur is the canonical next
    level, 1 not canonical, 2 a node whose signature differs from its block
    head's, 3 two blocks with equal signatures."""
    lib = _load()
    n = int(g.num_nodes)
    off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
    dst = np.ascontiguousarray(g.dst, dtype=np.uint32)
    lab = np.ascontiguousarray(g.edge_label)
    if lab.dtype != np.uint8:
        lab = np.ascontiguousarray(lab, dtype=np.uint32)
    p, c = _u32(prev), _u32(cur)
    if p.size != n or c.size != n:
        raise ValueError("level sizes disagree with the graph")
    cnt = np.zeros(1, np.uint64)
    bad = np.zeros(1, np.uint64)
    rc = lib.oracle_check_level(n, _ptr(off), _ptr(dst), _ptr(lab), 1 if lab.dtype == np.uint8 else 4,
                                _ptr(p), _ptr(c), int(threads or os.cpu_count() or 1),
                                cnt.ctypes.data_as(ctypes.c_void_p), bad.ctypes.data_as(ctypes.c_void_p))
    return int(rc), int(cnt[0]), int(bad[0])
