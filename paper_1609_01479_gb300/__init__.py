"""Binary-fluid D3Q19 lattice-Boltzmann step on one GB300 (sm_103a).

The hot path is hand-written CUDA behind the C ABI in include/ld.h; ``ld``
is its Python binding (argument marshalling only) and ``inputs`` builds the
seeded synthetic initial fields. Importing the package loads nothing: the
CUDA library is built/loaded on first use and every call raises if it is
unavailable (there is no CPU fallback).
"""

__all__ = ["ld", "inputs", "build"]
