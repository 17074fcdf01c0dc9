"""GB300-native Lagrangian grain-envelope particle solver (arXiv 2504.12858).

The compute path is the CUDA shared library built from ``csrc/`` (C ABI declared
in ``include/gp.h``); ``native`` is its thin ctypes binding and ``inputs`` the
seeded synthetic workloads.  Importing this package does not load the library;
``native.load()`` does, and raises if it has not been built.
"""
__all__ = ["inputs", "native"]
