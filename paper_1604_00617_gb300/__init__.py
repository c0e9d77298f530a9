"""GB300-native block cyclic reduction with hierarchically low-rank blocks
(Accelerated Cyclic Reduction).

The solver is the CUDA library ``_build/libacr.so`` behind the C ABI of
``include/acr.h``; :mod:`._lib` is its ctypes binding (same function names) and
:mod:`.solver` a small convenience layer over it.  Build the library with
:func:`build`.  Nothing here computes on the CPU.
"""

from .build import build  # noqa: F401

__all__ = ["build"]
