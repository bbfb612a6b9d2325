"""GPU maximum cardinality bipartite matching for GB300 (sm_103a).

The method is the augmenting-path algorithm of Deveci, Kaya, Ucar and
Catalyurek (arXiv 1303.1379): level-synchronous BFS from all unmatched
columns (GPUBFS / GPUBFS-WR), Alternate and FixMatching, repeated until no
augmenting path remains (APFB / APsB).  The compute path is the CUDA library
``libbmatch.so`` (C-ABI in include/bmatch.h); ``bmatch`` is its ctypes
binding and ``synth`` draws seeded synthetic inputs.

Importing the package loads nothing; ``bmatch.load()`` loads the library.
"""
__all__ = ["bmatch", "synth", "build"]
