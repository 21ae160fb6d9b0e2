"""GB300 (sm_103a) Wave-ADR multigrid library for the 2D Helmholtz equation.

The compute path is the CUDA library built from `csrc/` (C ABI in
include/wave_adr.h); `binding` is a thin ctypes layer over it.  Importing
the package does not load the library; `binding.load()` does, and raises if
it has not been built.
"""
from . import build  # noqa: F401

__all__ = ["build", "binding"]
