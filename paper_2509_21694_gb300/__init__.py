"""GB300-native energy-and-force evaluation of a depth-pruned message-passing
interatomic potential on large periodic systems split into halo partitions
(arXiv 2509.21694).

The compute path is the CUDA library ``libmpip.so`` (C ABI in
``include/mpip.h``); ``binding`` is its ctypes binding.  Import ``binding``
explicitly: it raises if the library has not been built.
"""

__all__ = ["binding", "build"]
