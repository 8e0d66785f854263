"""gbspmv: sparse matrix-vector multiplication in CRS and JDS storage on
GB300 (sm_103a), after Schubert, Hager & Fehske, "Performance limitations
for sparse matrix-vector multiplications on current multicore
environments".

The compute path is the CUDA library libgbspmv.so (C ABI in
include/gbspmv.h); this package only marshals arguments to it.  Importing
the package does not load the library; the first product does, and fails
loudly if it is missing.
"""
from __future__ import annotations

import importlib

__all__ = ["CRSMatrix", "JDSMatrix", "GbspError", "SpMVFunction", "power_apply", "Batch",
           "gather_sum", "HybridMatrix", "build", "synth"]

_LAZY = {
    "CRSMatrix": "sparse", "JDSMatrix": "sparse", "GbspError": "_lib",
    "SpMVFunction": "autograd", "power_apply": "autograd", "Batch": "batch",
    "gather_sum": "gather", "HybridMatrix": "sparse",
}


def build(force: bool = False) -> str:
    """Compile libgbspmv.so for sm_103a (in-tree)."""
    return importlib.import_module(".buildlib", __name__).build(force=force)


def __getattr__(name):
    if name in _LAZY:
        return getattr(importlib.import_module("." + _LAZY[name], __name__), name)
    if name == "synth":
        return importlib.import_module(".synth", __name__)
    raise AttributeError(name)
