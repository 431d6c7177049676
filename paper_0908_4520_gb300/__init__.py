"""GB300-native high-order lattice Boltzmann hot path (Meng & Zhang).

The compute lives in liblb.so (CUDA kernels for sm_103a behind the C-ABI of
include/lb.h).  ``capi`` is the ctypes binding with the C names; ``Lattice``
is a small object wrapper around one handle.  ``inputs`` holds the seeded
workload generators (no arithmetic of the method).  Nothing here computes
on the CPU.
"""
from __future__ import annotations

__all__ = ["Lattice", "Batch", "capi", "build"]


def build(force: bool = False) -> str:
    from .builder import build as _b

    return _b(force=force)


def __getattr__(name):
    import importlib

    if name == "capi":
        return importlib.import_module(".capi", __name__)
    if name == "Lattice":
        return importlib.import_module(".lattice", __name__).Lattice
    if name == "Batch":
        return importlib.import_module(".batch", __name__).Batch
    raise AttributeError(name)
