"""GB300-native cascaded bilateral sampling (CABS, arXiv 1607.07395).

The compute path lives in libcabs.so (CUDA for sm_103a, C ABI in
include/cabs.h); ``cabs`` is its Python binding. Importing this package does
not load the library; the first call does, and fails loudly if it is absent.
"""
from . import cabs  # noqa: F401

__all__ = ["cabs"]
