"""The 256M-node / 2B-edge graph (64-bit edge offsets, identifier array far
larger than L2).  The oracle cannot run at this size, so the result is checked
through properties that hold at any size, computed with torch on the device:
level 0 equals the oracle's level 0; every level is canonical, has the reported
number of blocks and refines the level before; and on sampled nodes, equal
identifiers <=> equal signatures, computed on the host from Definition 3.

Needs about 20 GB of host memory and a few minutes: runs only with
KBISIM_LARGE=1."""
import os

import numpy as np
import pytest

import oracle
from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim
from tests.gpu_util import signature

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("KBISIM_LARGE") != "1",
                                 reason="256M-node graph: set KBISIM_LARGE=1")]


def _check_level_on_device(torch, p, prev, count):
    n = p.numel()
    assert int(p.max()) + 1 == count
    first = torch.full((count,), n, dtype=torch.int64, device=p.device)
    first.scatter_reduce_(0, p.long(), torch.arange(n, device=p.device), reduce="amin")
    assert int(first.max()) < n, "a block id without a node"
    assert bool((first[1:] > first[:-1]).all()), "not canonical"
    if prev is not None:
        pair = (p.long() << 32) | prev.long()
        assert torch.unique(pair).numel() == count, "does not refine the previous level"
    return first


def test_large_graph_properties():
    torch = pytest.importorskip("torch")
    g = synth.config_large_single()
    with KBisim() as kb:
        res = kb.build(g, 10)
        lvl0 = np.empty(g.num_nodes, np.uint32)
        cnt0 = oracle._load().oracle_level0(g.num_nodes, g.node_label.ctypes.data, None, lvl0.ctypes.data)
        assert cnt0 == res.counts[0]
        prev_host = None
        prev_dev = None
        rng = np.random.default_rng(5)
        for lev in range(res.rounds_run + 1):
            host = kb.pids(lev)
            if lev == 0:
                assert np.array_equal(host, lvl0)
            p = torch.from_numpy(host.view(np.int32)).cuda()
            first = _check_level_on_device(torch, p, prev_dev, res.counts[lev]).cpu().numpy()
            if lev:
                sigs = {}
                for u in rng.choice(g.num_nodes, size=400, replace=False).tolist():
                    s = signature(g, prev_host, u)
                    assert signature(g, prev_host, int(first[host[u]])) == s, (lev, u)
                    sigs.setdefault(s, set()).add(int(host[u]))
                assert all(len(b) == 1 for b in sigs.values())
            prev_host, prev_dev = host, p
