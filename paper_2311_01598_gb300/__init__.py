"""GB300-native RNS hybrid key switching (CiFlow, arxiv 2311.01598).

The compute path lives in the CUDA shared library built from ``csrc/`` and
exposed through a C ABI (``include/ks.h``); ``ks`` is its thin ctypes binding.
Importing the package does not load the library; ``ks.lib()`` does, and
raises if it is missing.
"""
__all__ = ["inputs"]
