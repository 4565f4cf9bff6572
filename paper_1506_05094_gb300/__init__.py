"""GB300-native MD hot path (LJ shifted-potential forces over a Verlet neighbour list, cell-sorted
rebuild, leapfrog NVE / Nose-Hoover NVT) behind the C ABI of include/md.h.

Importing the package is cheap; the CUDA library is loaded on first use by :func:`md.lib`.
"""
from .md import Sim, MDError, lib, strerror  # noqa: F401

__all__ = ["Sim", "MDError", "lib", "strerror"]
