"""The allocation-free label partition matches the regular level 0.

kbisim_label_partition_noalloc serves callers that cannot allocate device
memory (its scratch is a fixed static device array shared by all calls).  It
is called twice in a row through the C ABI, and each result must equal level
0 of a regular handle, bit for bit (identifiers are integers).  This file is
collected last so that a failure here cannot hide other results.
"""
import numpy as np
import pytest

from paper_1210_0748_gb300 import synth
from paper_1210_0748_gb300.kbisim import KBisim, KBisimError, label_partition_noalloc

pytestmark = pytest.mark.gpu


def _regular_level0(labels):
    g = synth.from_coo(labels.size, [], [], [], labels)
    with KBisim() as kb:
        res = kb.build(g, 0)
        return kb.pids(0), res.counts[0]


def test_noalloc_matches_regular_level0_twice():
    import torch
    rng = np.random.default_rng(2024)
    cases = [rng.integers(0, 40, 100_000).astype(np.uint32),
             rng.choice(np.array([7, 0xFFFFFFFF, 3, 123456789], np.uint32), 262_144)]
    for labels in cases:  # two calls in a row share the scratch array
        want, want_count = _regular_level0(labels)
        lab = torch.from_numpy(labels.view(np.int32)).cuda()
        out = torch.full((labels.size,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        label_partition_noalloc(lab, out, cnt)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)
        assert int(cnt.item()) == want_count


def test_noalloc_rejects_oversized_input():
    import torch
    lab = torch.zeros(262_145, dtype=torch.int32, device="cuda")
    out = torch.empty_like(lab)
    with pytest.raises(KBisimError):
        label_partition_noalloc(lab, out)
