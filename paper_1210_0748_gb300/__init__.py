"""GB300-native k-bisimulation partition refinement.

The computation lives in libkbisim.so (CUDA kernels for sm_103a behind the C
ABI of include/kbisim.h).  ``kbisim.KBisim`` is the Python binding;
``synth`` draws seeded synthetic graphs; ``build`` compiles the library.
"""
from .kbisim import KBisim, KBisimError, Result, load_library  # noqa: F401

__all__ = ["KBisim", "KBisimError", "Result", "load_library"]
