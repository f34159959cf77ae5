"""B300-native QAOA max-cut state-vector simulator (sm_103a CUDA kernels behind a C ABI).

``paper_2312_03019_b300.inputs`` (seeded graphs and angles) imports without the CUDA library.
Every other name resolves lazily from ``paper_2312_03019_b300.binding``, which loads
``libqaoa_b300.so`` and fails loudly when it is missing.
"""
from __future__ import annotations

import importlib

__all__ = ["inputs", "binding"]


def __getattr__(name):
    if name in ("inputs", "binding", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    mod = importlib.import_module(f"{__name__}.binding")
    try:
        return getattr(mod, name)
    except AttributeError as e:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from e
