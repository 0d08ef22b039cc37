"""B300 firing runtime for PRUNE dynamic, decidable dataflow graphs.

The compute path is libprune.so (CUDA, sm_103a) behind the C ABI of
include/prune.h; ``graph.Graph`` and the single-actor helpers marshal
arguments to it.  ``synth`` draws the seeded synthetic workloads.
Submodules are imported lazily so that the generator works without the
library.
"""
__all__ = ["graph", "synth", "build"]
