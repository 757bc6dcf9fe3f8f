"""GB300-native pseudopotential LBM for boiling heat transfer (arXiv 2201.04560).

The compute path is libppl.so (hand-written sm_103a CUDA behind the C ABI of
include/ppl.h); this package is a thin ctypes binding with the same entry points.
"""
from .ppl import (PplError, Simulation, library_path, load_library, maxwell, refine_a, tc)  # noqa: F401

__all__ = ["PplError", "Simulation", "library_path", "load_library", "maxwell", "refine_a", "tc"]
