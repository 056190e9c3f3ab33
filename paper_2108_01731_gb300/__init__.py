"""GB300-native LambdaCC best-move / contraction path (arXiv 2108.01731).

The compute path lives in ``liblcc.so`` (hand-written sm_103a CUDA behind a
C ABI declared in ``include/lcc.h``); ``lcc`` is its thin ctypes binding and
``inputs`` the seeded synthetic-graph generators.  Importing the package does
not load the CUDA library; ``lcc.load()`` does, and fails loudly if it has not
been built.
"""
__all__ = ["lcc", "inputs"]
