"""The C ABI library loads and exports every entry point include/kbisim.h
declares (no GPU needed: nothing here computes)."""
import ctypes
import os
import re

from paper_1210_0748_gb300 import build as kbuild
from paper_1210_0748_gb300 import kbisim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "kbisim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kbisim_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("kbisim_create", "kbisim_build", "kbisim_update", "kbisim_extend", "kbisim_pids",
                 "kbisim_pids_device", "kbisim_last_error", "kbisim_destroy", "kbisim_refine",
                 "kbisim_load"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = kbuild.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding knows every declared function
    assert set(declared_functions()) <= set(kbisim.SIGNATURES)


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    try:
        kbisim.KBisim()
    except kbisim.KBisimError as e:
        assert e.code == kbisim.ERR_CUDA
    else:  # pragma: no cover
        raise AssertionError("created a handle without a GPU")


def test_binding_rejects_bad_tensors_before_the_library():
    """The binding checks device buffers (CUDA, current device, int32,
    contiguous, large enough) before any pointer reaches the library; these
    checks run on the host, so they are tested on the CPU."""
    import pytest
    import torch
    ok = torch.zeros(4, dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        kbisim.label_partition_noalloc(ok, ok)
    with pytest.raises(ValueError, match="torch tensor"):
        kbisim.label_partition_noalloc([0, 1], ok)
    with pytest.raises(ValueError):
        kbisim.check_device_tensor(torch.zeros(4, dtype=torch.int64), "x", 1)
    with pytest.raises(ValueError):
        kbisim.check_device_tensor(ok, "x", 8)
