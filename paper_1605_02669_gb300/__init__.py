"""GB300 (sm_103a) synchronous-step Ant Colony System (Skinderowicz, JPDC 2016).

The compute path is libacs.so (CUDA, C ABI in include/acs.h); ``acs`` is its
ctypes binding and ``instances`` draws seeded synthetic TSP instances.
"""
from . import instances  # noqa: F401
