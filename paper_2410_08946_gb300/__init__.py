"""GB300-native watershed and waterfall partitioning (arXiv 2410.08946).

The compute path is the C-ABI library ``libws.so`` (hand-written CUDA for
sm_103a, declared in ``include/ws.h``); ``binding`` is its thin ctypes
wrapper.  ``synth`` holds the seeded input generators.  Importing the package
loads nothing; the CUDA library is loaded on first use of ``binding``.
"""
__all__ = ["binding", "synth"]
