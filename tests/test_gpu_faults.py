"""Failure handling through the C ABI: a failed call leaves the previous
result readable (the header's promise), checked mode reports a bad index
before any kernel uses it, and the budget is enforced by the library.

Every failure is made on the host (the library's KBISIM_FAULT_* test hooks,
or a small HBM budget): an allocation that reports failure, a round that
reports a timeout, or (checked mode only) one stored edge target set to
num_nodes, one past the last node, which the index check must report.  None
of them makes a kernel fault or wait."""
import os

import numpy as np
import pytest

from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import (ERR_BUDGET, ERR_CHECKED, ERR_OUT_OF_MEMORY, ERR_STATE,
                                          ERR_TIMEOUT, KBisim, KBisimError)
from tests.gpu_util import assert_same, oracle_levels

pytestmark = pytest.mark.gpu


@pytest.fixture
def env():
    """Sets KBISIM_FAULT_* variables for one block and always clears them."""
    keys = []

    class Env:
        def set(self, **kv):
            for k, v in kv.items():
                os.environ[k] = str(v)
                keys.append(k)

        def clear(self):
            for k in keys:
                os.environ.pop(k, None)

    e = Env()
    yield e
    e.clear()


def _graph():
    # 5000 nodes: level buffers are not a multiple of the 2 MB allocation
    # granule, so even an unchecked read one past the end would stay inside it
    return synth.config_single_large(scale=5000 / 16_000_000, seed=77)


def _snapshot(kb, k):
    return kb.all_pids(k)


def test_failed_refine_keeps_previous_levels(env):
    g = _graph()
    ref3 = oracle_levels(g, 3, early_stop=False)
    with KBisim(early_stop=False) as kb:
        res = kb.build(g, 3)
        before = _snapshot(kb, 3)
        assert_same(res, before, ref3)
        env.set(KBISIM_FAULT_ALLOC=0)
        with pytest.raises(KBisimError) as e:
            kb.refine(6)
        assert e.value.code == ERR_OUT_OF_MEMORY
        env.clear()
        assert np.array_equal(_snapshot(kb, 3), before)
        env.set(KBISIM_FAULT_TIMEOUT_ROUND=2)
        with pytest.raises(KBisimError) as e:
            kb.refine(5)
        assert e.value.code == ERR_TIMEOUT
        env.clear()
        assert np.array_equal(_snapshot(kb, 3), before)
        with pytest.raises(KBisimError):
            kb.pids(4)  # the failed call's k was never taken on
        res6 = kb.refine(6)
        assert_same(res6, kb.all_pids(6), oracle_levels(g, 6, early_stop=False))


def test_failed_extend_keeps_previous_levels(env):
    g = _graph()
    with KBisim(early_stop=False) as kb:
        kb.build(g, 1)
        before = _snapshot(kb, 1)
        env.set(KBISIM_FAULT_TIMEOUT_ROUND=3)
        with pytest.raises(KBisimError) as e:
            kb.extend(5)
        assert e.value.code == ERR_TIMEOUT
        env.clear()
        assert np.array_equal(_snapshot(kb, 1), before)
        r = kb.extend(5)
        assert_same(r, kb.all_pids(5), oracle_levels(g, 5, early_stop=False))


def test_budget_is_enforced_and_keeps_previous_levels():
    g = _graph()
    with KBisim(early_stop=False, hbm_budget_bytes=1 << 40) as probe:
        probe.build(g, 2)
        need = probe.device_bytes
    assert need > 0
    with KBisim(early_stop=False, hbm_budget_bytes=need + 4096) as kb:
        kb.build(g, 2)
        assert kb.device_bytes <= need + 4096
        before = _snapshot(kb, 2)
        with pytest.raises(KBisimError) as e:
            kb.refine(200)  # 198 more levels do not fit, even without the idle scratch
        assert e.value.code == ERR_BUDGET
        assert np.array_equal(_snapshot(kb, 2), before)
        assert kb.device_bytes <= need + 4096
    with KBisim(hbm_budget_bytes=1 << 20) as kb:
        with pytest.raises(KBisimError) as e:
            kb.build(synth.config_single_large(scale=1 / 256, seed=3), 3)
        assert e.value.code == ERR_BUDGET


def test_budget_drops_idle_scratch_before_failing():
    """A handle keeps its scratch between calls (the staging of its load,
    here); when a call needs more than the budget allows, the scratch no
    running step uses is released first, so the call succeeds."""
    g = _graph()
    with KBisim(early_stop=False) as kb:
        kb.build(g, 2)
        kb.refine(2)  # the levels the build made become this call's spares
        held = kb.device_bytes
        kb.refine(2)
        assert kb.device_bytes == held  # a repeated call allocates nothing
        kb.set_hbm_budget(held)
        res = kb.refine(3)  # one more level: fits once the load's staging is gone
        assert kb.device_bytes <= held
        assert_same(res, kb.all_pids(3), oracle_levels(g, 3, early_stop=False))


def test_checked_mode_reports_a_bad_index(env):
    g = _graph()
    with KBisim(checked=True) as kb:
        res = kb.build(g, 4)
        before = _snapshot(kb, 4)
        assert_same(res, before, oracle_levels(g, 4))
        env.set(KBISIM_FAULT_CORRUPT_DST=1)
        with pytest.raises(KBisimError) as e:
            kb.refine(4)
        assert e.value.code == ERR_CHECKED
        env.clear()
        assert np.array_equal(_snapshot(kb, 4), before)
        res = kb.refine(4)  # the target was put back
        assert_same(res, kb.all_pids(4), oracle_levels(g, 4))
    with KBisim(checked=False) as kb:  # the hook is inert without checked mode
        env.set(KBISIM_FAULT_CORRUPT_DST=1)
        res = kb.build(g, 4)
        env.clear()
        assert_same(res, kb.all_pids(4), oracle_levels(g, 4))


def test_update_failure_after_the_batch_is_stored(env):
    """The recomputing update (maintain=False): a round that fails after the
    batch was stored leaves the updated graph without levels."""
    from oracle.update import MultiGraph
    g = _graph()
    mg = MultiGraph(g.num_nodes, g.node_label, g.src(), g.dst, g.edge_label)
    ins = (np.array([1, 2], np.uint32), np.array([3, 4], np.uint32), np.array([0, 1], np.uint32))
    with KBisim(maintain=False) as kb:
        kb.build(g, 3)
        env.set(KBISIM_FAULT_TIMEOUT_ROUND=1)
        with pytest.raises(KBisimError) as e:
            kb.update(3, ins=ins)
        assert e.value.code == ERR_TIMEOUT
        env.clear()
        with pytest.raises(KBisimError) as e:
            kb.pids(0)
        assert e.value.code == ERR_STATE
        mg.apply(ins=list(zip(*ins)))
        res = kb.refine(3)
        assert_same(res, kb.all_pids(3), mg.kbisim(3))
