"""GB300-native TLMPM cutting hot path (BladeMaster, arXiv 2609.27342).

The substep -- side labels, stress, label-masked P2G, coupled grid update
with tool and pair contact, G2P/MUSL/F update -- runs in hand-written sm_103a
kernels behind the C ABI of include/blademaster.h.  This package is the thin
Python binding: ``Scene`` (one scene, plain per-kernel launches) and
``Batch`` (many uneven scenes, CUDA-graph launches).
"""
from ._abi import BMError, load, library_path  # noqa: F401
from .sim import Batch, Scene, TorchAllocator, footprint  # noqa: F401

__all__ = ["Scene", "Batch", "TorchAllocator", "BMError", "load", "library_path", "footprint"]
