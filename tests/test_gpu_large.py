"""The 256M-node / 2B-edge graph (64-bit edge offsets, identifier array far
larger than L2).  The oracle (ordered maps on one core) would need most of an
hour here, so every level is checked against its definition instead:
level 0 equals the oracle's level 0, and each later level passes the
Proposition 2 checker (oracle/check_levels.cpp: canonical numbering, every
node carries its block head's signature, different blocks have different
signatures, signatures built exactly from the previous level on the host).

Runs wherever the host has the memory for it (about 40 GB: the graph, two
levels and the checker's fingerprints) and the GPU about 100 GB free."""
import os

import numpy as np
import pytest

import oracle
from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim

pytestmark = pytest.mark.gpu

HOST_BYTES = 64 << 30
DEVICE_BYTES = 100 << 30


def _host_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def test_large_graph_levels_pass_the_checker():
    torch = pytest.importorskip("torch")
    if _host_available() < HOST_BYTES:
        pytest.skip("needs %d GiB of free host memory" % (HOST_BYTES >> 30))
    if torch.cuda.mem_get_info()[0] < DEVICE_BYTES:
        pytest.skip("needs %d GiB of free device memory" % (DEVICE_BYTES >> 30))
    g = synth.config_large_single()
    with KBisim() as kb:
        res = kb.build(g, 10)
        assert res.rounds_run >= 2
        lvl0 = np.empty(g.num_nodes, np.uint32)
        cnt0 = oracle._load().oracle_level0(g.num_nodes, g.node_label.ctypes.data, None, lvl0.ctypes.data)
        prev = kb.pids(0)
        assert cnt0 == res.counts[0]
        assert np.array_equal(prev, lvl0)
        del lvl0
        threads = max(1, min(64, os.cpu_count() or 1))
        for lev in range(1, res.rounds_run + 1):
            cur = kb.pids(lev)
            code, blocks, bad = oracle.check_level(g, prev, cur, threads=threads)
            assert code == 0, "level %d: checker code %d at node %d" % (lev, code, bad)
            assert blocks == res.counts[lev]
            prev = cur
        assert res.counts[res.rounds_run] == res.counts[res.rounds_run - 1] or res.rounds_run == 10
