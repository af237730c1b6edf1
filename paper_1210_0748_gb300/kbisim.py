"""Python binding of libkbisim (ctypes over the C ABI in include/kbisim.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory (for inputs and
outputs that live on the GPU) and the CUDA stream.  If the library is not
built, or no GPU is usable, these calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkbisim.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_OUT_OF_MEMORY = 2
ERR_BUDGET = 3
ERR_CUDA = 4
ERR_TIMEOUT = 5
ERR_CHECKED = 6
ERR_STATE = 7
DELETED = 0xFFFFFFFF
MAX_K = 1024

KERNEL_NAMES = ["label_group", "sig_small", "sig_medium", "sig_hub", "group", "verify",
                "renumber", "other"]

_ERR_NAMES = {ERR_INVALID_ARG: "INVALID_ARG", ERR_OUT_OF_MEMORY: "OUT_OF_MEMORY",
              ERR_BUDGET: "BUDGET", ERR_CUDA: "CUDA", ERR_TIMEOUT: "TIMEOUT",
              ERR_CHECKED: "CHECKED", ERR_STATE: "STATE"}


class KBisimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_uint64), ("early_stop", ctypes.c_int),
                ("hash_seed", ctypes.c_uint64), ("hash_bits", ctypes.c_uint32),
                ("checked", ctypes.c_int), ("collect_timing", ctypes.c_int), ("maintain", ctypes.c_int),
                ("hub_bucket_keys", ctypes.c_uint32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_uint64), ("num_edges", ctypes.c_uint64),
                ("node_label", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("edge_label", ctypes.c_void_p), ("edge_label_bytes", ctypes.c_uint32),
                ("on_device", ctypes.c_int)]


class ResultDesc(ctypes.Structure):
    _fields_ = [("k_requested", ctypes.c_uint32), ("rounds_run", ctypes.c_uint32),
                ("block_count", ctypes.POINTER(ctypes.c_uint64))]


class BatchDesc(ctypes.Structure):
    _fields_ = [("add_node_label", ctypes.c_void_p), ("n_add_nodes", ctypes.c_uint64),
                ("ins_src", ctypes.c_void_p), ("ins_dst", ctypes.c_void_p),
                ("ins_label", ctypes.c_void_p), ("n_ins", ctypes.c_uint64),
                ("del_src", ctypes.c_void_p), ("del_dst", ctypes.c_void_p),
                ("del_label", ctypes.c_void_p), ("n_del", ctypes.c_uint64),
                ("del_nodes", ctypes.c_void_p), ("n_del_nodes", ctypes.c_uint64),
                ("on_device", ctypes.c_int)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double * 8), ("launches", ctypes.c_uint64 * 8)]


class UpdateInfo(ctypes.Structure):
    _fields_ = [("incremental", ctypes.c_int), ("reason", ctypes.c_int),
                ("frontier_nodes", ctypes.c_uint64), ("levels", ctypes.c_uint64), ("in_place", ctypes.c_int)]


MAINT_REASONS = {0: "incremental", 1: "off", 2: "no_store", 3: "frontier", 4: "capacity", 5: "deletes", 6: "cost"}


class RoundStats(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_uint64), ("unique_keys", ctypes.c_uint64),
                ("max_signature", ctypes.c_uint64), ("collided_nodes", ctypes.c_uint64),
                ("hub_nodes", ctypes.c_uint64)]


_lib = None

# exported symbols and their signatures (checked by the CPU tests)
SIGNATURES = {
    "kbisim_default_options": (None, [ctypes.POINTER(Options)]),
    "kbisim_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Options)]),
    "kbisim_destroy": (None, [ctypes.c_void_p]),
    "kbisim_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "kbisim_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GraphDesc)]),
    "kbisim_refine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ResultDesc)]),
    "kbisim_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.c_uint32,
                                    ctypes.POINTER(ResultDesc)]),
    "kbisim_extend": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ResultDesc)]),
    "kbisim_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchDesc), ctypes.c_uint32,
                                     ctypes.POINTER(ResultDesc), ctypes.POINTER(ctypes.c_uint64)]),
    "kbisim_pids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int]),
    "kbisim_pids_device": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_uint32]),
    "kbisim_num_nodes": (ctypes.c_uint64, [ctypes.c_void_p]),
    "kbisim_num_edges": (ctypes.c_uint64, [ctypes.c_void_p]),
    "kbisim_device_bytes": (ctypes.c_uint64, [ctypes.c_void_p]),
    "kbisim_hub_bucket_keys": (ctypes.c_uint32, [ctypes.c_void_p]),
    "kbisim_get_update_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(UpdateInfo)]),
    "kbisim_set_hbm_budget": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "kbisim_get_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KernelTimes)]),
    "kbisim_reset_times": (None, [ctypes.c_void_p]),
    "kbisim_get_round_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32,
                                              ctypes.POINTER(RoundStats)]),
    "kbisim_label_partition_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                                      ctypes.c_void_p, ctypes.c_void_p]),
    "kbisim_build_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.c_void_p,
                                         ctypes.c_uint32, ctypes.c_void_p]),
    "kbisim_many_pids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_int]),
    "kbisim_many_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.c_void_p]),
}


def concat_graphs(graphs):
    """Disjoint union of CSR graphs for ``kbisim_build_many``: node ids of graph
    j shifted by the nodes before it.  Returns (graph, node starts [G+1])."""
    from .synth import Graph
    n = np.array([g.num_nodes for g in graphs], dtype=np.int64)
    m = np.array([g.num_edges for g in graphs], dtype=np.int64)
    starts = np.zeros(len(graphs) + 1, dtype=np.uint64)
    starts[1:] = np.cumsum(n)
    ebase = np.zeros(len(graphs) + 1, dtype=np.int64)
    ebase[1:] = np.cumsum(m)
    wide = any(g.edge_label.dtype != np.uint8 for g in graphs)
    off = np.empty(int(starts[-1]) + 1, dtype=np.uint64)
    dst = np.empty(int(ebase[-1]), dtype=np.uint32)
    lab = np.empty(int(ebase[-1]), dtype=np.uint32 if wide else np.uint8)
    nl = np.empty(int(starts[-1]), dtype=np.uint32)
    for j, g in enumerate(graphs):
        a, b = int(starts[j]), int(starts[j + 1])
        off[a:b] = g.offsets[:-1].astype(np.uint64) + np.uint64(ebase[j])
        dst[ebase[j]:ebase[j + 1]] = g.dst.astype(np.uint32) + np.uint32(a)
        lab[ebase[j]:ebase[j + 1]] = g.edge_label
        nl[a:b] = g.node_label
    off[-1] = np.uint64(ebase[-1])
    return Graph(int(starts[-1]), off, dst, lab, nl), starts


def load_library(path: str = LIB_PATH):
    """Load libkbisim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libkbisim.so is not built (run paper_1210_0748_gb300/build.py)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


class _Pinned:
    """Keeps host arrays alive for the duration of a call."""

    def __init__(self):
        self.keep = []

    def host(self, a, dtype):
        arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
        self.keep.append(arr)
        return arr.ctypes.data if arr.size else None, arr

    def dev(self, t, dtype):
        torch = _torch()
        tt = t.to(dtype).contiguous()
        self.keep.append(tt)
        return tt.data_ptr() if tt.numel() else None, tt


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except Exception:  # pragma: no cover
        return False


class Result:
    def __init__(self, desc: ResultDesc):
        self.k_requested = int(desc.k_requested)
        self.rounds_run = int(desc.rounds_run)
        self.counts = [int(desc.block_count[i]) for i in range(self.k_requested + 1)]

    def __repr__(self):
        return "Result(k=%d, rounds_run=%d, counts=%s)" % (self.k_requested, self.rounds_run, self.counts)


class KBisim:
    """One library handle: a device-resident graph and its partition levels."""

    def __init__(self, device: int = 0, stream=None, early_stop: bool = True,
                 hash_seed: int = 0x12100748, hash_bits: int = 64, checked: bool = False,
                 collect_timing: bool = False, hbm_budget_bytes: int = 0, maintain=True,
                 hub_bucket_keys: int = 0):
        lib = load_library()
        self._lib = lib
        opt = Options()
        lib.kbisim_default_options(ctypes.byref(opt))
        if stream is None:
            try:
                torch = _torch()
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        opt.stream = stream or None
        opt.device = device
        opt.early_stop = 1 if early_stop else 0
        opt.hash_seed = hash_seed & 0xFFFFFFFFFFFFFFFF
        opt.hash_bits = hash_bits
        opt.checked = 1 if checked else 0
        opt.collect_timing = 1 if collect_timing else 0
        opt.hbm_budget_bytes = hbm_budget_bytes
        # False/0: recompute; True/1: frontier path while it measures cheaper;
        # "always"/2: frontier path whenever it applies
        opt.maintain = 2 if maintain in ("always", 2) else (1 if maintain else 0)
        opt.hub_bucket_keys = int(hub_bucket_keys)
        h = ctypes.c_void_p()
        rc = lib.kbisim_create(ctypes.byref(h), ctypes.byref(opt))
        if rc != OK:
            raise KBisimError(rc, "kbisim_create failed")
        self._h = h
        self.device = device
        self.stream = stream

    # -- helpers --------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            msg = self._lib.kbisim_last_error(self._h)
            raise KBisimError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kbisim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- graph ----------------------------------------------------------------
    def _graph_desc(self, keep: _Pinned, num_nodes, node_label, dst, edge_label, offsets=None,
                    src=None):
        g = GraphDesc()
        g.num_nodes = int(num_nodes)
        on_dev = _is_torch(dst) and dst.is_cuda
        g.on_device = 1 if on_dev else 0
        torch = _torch() if on_dev else None
        if on_dev:
            g.node_label, _ = keep.dev(node_label, torch.int32)
            g.dst, dt = keep.dev(dst, torch.int32)
            g.num_edges = dt.numel()
            if offsets is not None:
                g.offsets, _ = keep.dev(offsets, torch.int64)
            else:
                g.src, _ = keep.dev(src, torch.int32)
            el = edge_label
            if el.dtype == torch.uint8:
                g.edge_label, _ = keep.dev(el, torch.uint8)
                g.edge_label_bytes = 1
            else:
                g.edge_label, _ = keep.dev(el, torch.int32)
                g.edge_label_bytes = 4
        else:
            g.node_label, _ = keep.host(node_label, np.uint32)
            g.dst, dt = keep.host(dst, np.uint32)
            g.num_edges = dt.size
            if offsets is not None:
                g.offsets, _ = keep.host(offsets, np.uint64)
            else:
                g.src, _ = keep.host(src, np.uint32)
            el = np.asarray(edge_label)
            if el.dtype == np.uint8:
                g.edge_label, _ = keep.host(el, np.uint8)
                g.edge_label_bytes = 1
            elif el.dtype == np.uint16:
                g.edge_label, _ = keep.host(el, np.uint16)
                g.edge_label_bytes = 2
            else:
                g.edge_label, _ = keep.host(el, np.uint32)
                g.edge_label_bytes = 4
        return g

    def load(self, graph=None, *, num_nodes=None, node_label=None, dst=None, edge_label=None,
             offsets=None, src=None):
        """Load a graph: a ``synth.Graph`` (CSR, host) or explicit arrays
        (numpy / host tensors, or CUDA tensors for an on-device load)."""
        keep = _Pinned()
        if graph is not None:
            g = self._graph_desc(keep, graph.num_nodes, graph.node_label, graph.dst,
                                 graph.edge_label, offsets=graph.offsets)
        else:
            g = self._graph_desc(keep, num_nodes, node_label, dst, edge_label, offsets=offsets,
                                 src=src)
        self._check(self._lib.kbisim_load(self._h, ctypes.byref(g)))

    def build_many(self, graphs, ks, *, union=None):
        """Batched build of independent graphs (``synth.Graph`` list) with
        k = ks[j] for graph j, all refined together.  ``union`` may pass the
        already concatenated graph and its node starts (``concat_graphs``).
        Results per graph: ``many_pids(j, level)``, ``many_info(j)``."""
        g_all, starts = union if union is not None else concat_graphs(graphs)
        keep = _Pinned()
        g = self._graph_desc(keep, g_all.num_nodes, g_all.node_label, g_all.dst, g_all.edge_label,
                             offsets=g_all.offsets)
        st = np.ascontiguousarray(np.asarray(starts, dtype=np.uint64))
        kk = np.ascontiguousarray(np.asarray(ks, dtype=np.uint32))
        if kk.size != st.size - 1:
            raise ValueError("need one k per graph")
        self._check(self._lib.kbisim_build_many(self._h, ctypes.byref(g), st.ctypes.data, int(kk.size),
                                                kk.ctypes.data))
        self._many_sizes = np.diff(st.astype(np.int64))
        self._many_k = kk.copy()

    def many_pids(self, j: int, level: int) -> np.ndarray:
        sizes = getattr(self, "_many_sizes", None)
        n = int(sizes[j]) if sizes is not None and 0 <= j < sizes.size else 0
        out = np.empty(max(n, 1), dtype=np.uint32)
        self._check(self._lib.kbisim_many_pids(self._h, int(j), int(level), out.ctypes.data, 0))
        return out[:n]

    def many_info(self, j: int):
        """(rounds_run, block counts of levels 0..k_j) of graph j."""
        r = ctypes.c_uint32(0)
        self._check(self._lib.kbisim_many_info(self._h, int(j), ctypes.byref(r), None))
        counts = np.zeros(int(self._many_k[j]) + 1, dtype=np.uint64)
        self._check(self._lib.kbisim_many_info(self._h, int(j), ctypes.byref(r), counts.ctypes.data))
        return int(r.value), counts

    def refine(self, k: int) -> Result:
        r = ResultDesc()
        self._check(self._lib.kbisim_refine(self._h, int(k), ctypes.byref(r)))
        return Result(r)

    def build(self, graph=None, k: int = 0, **arrays) -> Result:
        keep = _Pinned()
        if graph is not None:
            g = self._graph_desc(keep, graph.num_nodes, graph.node_label, graph.dst,
                                 graph.edge_label, offsets=graph.offsets)
        else:
            g = self._graph_desc(keep, arrays["num_nodes"], arrays["node_label"], arrays["dst"],
                                 arrays["edge_label"], offsets=arrays.get("offsets"),
                                 src=arrays.get("src"))
        r = ResultDesc()
        self._check(self._lib.kbisim_build(self._h, ctypes.byref(g), int(k), ctypes.byref(r)))
        return Result(r)

    def extend(self, k_new: int) -> Result:
        r = ResultDesc()
        self._check(self._lib.kbisim_extend(self._h, int(k_new), ctypes.byref(r)))
        return Result(r)

    def update(self, k: int, add_node_label=(), ins=(), dels=(), del_nodes=()):
        """Apply a maintenance batch (host arrays) and recompute levels 0..k.
        ins / dels: (src, dst, label) array triples.  Returns (Result, missing)."""
        keep = _Pinned()
        b = BatchDesc()
        b.add_node_label, a = keep.host(add_node_label, np.uint32)
        b.n_add_nodes = a.size
        if len(ins):
            s, d, l = ins
            b.ins_src, sa = keep.host(s, np.uint32)
            b.ins_dst, _ = keep.host(d, np.uint32)
            b.ins_label, _ = keep.host(l, np.uint32)
            b.n_ins = sa.size
        if len(dels):
            s, d, l = dels
            b.del_src, sa = keep.host(s, np.uint32)
            b.del_dst, _ = keep.host(d, np.uint32)
            b.del_label, _ = keep.host(l, np.uint32)
            b.n_del = sa.size
        b.del_nodes, dn = keep.host(del_nodes, np.uint32)
        b.n_del_nodes = dn.size
        b.on_device = 0
        r = ResultDesc()
        miss = ctypes.c_uint64(0)
        self._check(self._lib.kbisim_update(self._h, ctypes.byref(b), int(k), ctypes.byref(r),
                                            ctypes.byref(miss)))
        return Result(r), int(miss.value)

    # -- results ----------------------------------------------------------------
    @property
    def num_nodes(self) -> int:
        return int(self._lib.kbisim_num_nodes(self._h))

    @property
    def num_edges(self) -> int:
        return int(self._lib.kbisim_num_edges(self._h))

    @property
    def hub_bucket_keys(self) -> int:
        """Hub bucket size in use (fixed by the option, or tuned)."""
        return int(self._lib.kbisim_hub_bucket_keys(self._h))

    @property
    def device_bytes(self) -> int:
        """Device bytes the handle holds (what hbm_budget_bytes bounds)."""
        return int(self._lib.kbisim_device_bytes(self._h))

    def set_hbm_budget(self, nbytes: int) -> None:
        """Bound the device bytes later calls may hold (0 = no bound)."""
        self._check(self._lib.kbisim_set_hbm_budget(self._h, int(nbytes)))

    def pids(self, level: int, out=None):
        """Level ``level`` as a host numpy uint32 array, or into ``out`` (a CUDA
        int32 tensor of num_nodes elements)."""
        n = self.num_nodes
        if out is not None:
            check_device_tensor(out, "out", n, device=self.device)
            self._check(self._lib.kbisim_pids(self._h, int(level), ctypes.c_void_p(out.data_ptr()), 1))
            return out
        host = np.empty(n, dtype=np.uint32)
        self._check(self._lib.kbisim_pids(self._h, int(level),
                                          host.ctypes.data if n else None, 0))
        return host

    def pids_device_ptr(self, level: int) -> Optional[int]:
        p = self._lib.kbisim_pids_device(self._h, int(level))
        return int(p) if p else None

    def all_pids(self, k: int) -> np.ndarray:
        return np.stack([self.pids(i) for i in range(k + 1)]) if self.num_nodes else \
            np.zeros((k + 1, 0), np.uint32)

    def kernel_times(self) -> dict:
        kt = KernelTimes()
        self._check(self._lib.kbisim_get_kernel_times(self._h, ctypes.byref(kt)))
        return {name: (float(kt.total_ms[i]), int(kt.launches[i]))
                for i, name in enumerate(KERNEL_NAMES)}

    def reset_times(self):
        self._lib.kbisim_reset_times(self._h)

    def update_info(self) -> dict:
        """How the last update ran: incremental (frontier path) or recomputed,
        the reason for a recomputation, and the nodes signed over the levels."""
        ui = UpdateInfo()
        self._check(self._lib.kbisim_get_update_info(self._h, ctypes.byref(ui)))
        return {"incremental": bool(ui.incremental), "reason": MAINT_REASONS.get(int(ui.reason), str(ui.reason)),
                "frontier_nodes": int(ui.frontier_nodes), "levels": int(ui.levels),
                "in_place": bool(ui.in_place)}

    def round_stats(self, r: int) -> dict:
        st = RoundStats()
        self._check(self._lib.kbisim_get_round_stats(self._h, int(r), ctypes.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in RoundStats._fields_}


def check_device_tensor(t, name: str, min_numel: int, device=None) -> None:
    """Raise ValueError unless ``t`` is a contiguous CUDA int32 tensor on
    ``device`` (default: the current CUDA device) with at least ``min_numel``
    elements.  Runs before any pointer reaches the library, so a host tensor,
    a wrong dtype or a short buffer never becomes an out-of-range device write."""
    if not _is_torch(t):
        raise ValueError("%s must be a torch tensor" % name)
    torch = _torch()
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    want = torch.cuda.current_device() if device is None else int(device)
    if t.device.index != want:
        raise ValueError("%s is on cuda:%s, expected cuda:%d" % (name, t.device.index, want))
    if t.dtype != torch.int32:
        raise ValueError("%s must be int32, got %s" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < min_numel:
        raise ValueError("%s has %d elements, needs at least %d" % (name, t.numel(), min_numel))


def label_partition_noalloc(node_label, pid0, block_count=None, stream=None) -> None:
    """Level 0 of CUDA int32 tensor ``node_label`` into CUDA int32 tensor
    ``pid0`` (and the block count into a one-element CUDA int32 tensor),
    without any device allocation: see kbisim_label_partition_noalloc."""
    if not _is_torch(node_label):
        raise ValueError("node_label must be a torch tensor")
    check_device_tensor(node_label, "node_label", 0)
    check_device_tensor(pid0, "pid0", node_label.numel())
    if block_count is not None:
        check_device_tensor(block_count, "block_count", 1)
    lib = load_library()
    if stream is None:
        stream = _torch().cuda.current_stream().cuda_stream
    rc = lib.kbisim_label_partition_noalloc(
        ctypes.c_void_p(node_label.data_ptr()), node_label.numel(), ctypes.c_void_p(pid0.data_ptr()),
        ctypes.c_void_p(block_count.data_ptr()) if block_count is not None else None,
        ctypes.c_void_p(stream) if stream else None)
    if rc != OK:
        raise KBisimError(rc, "kbisim_label_partition_noalloc failed")
