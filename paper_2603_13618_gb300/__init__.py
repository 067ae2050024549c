"""GB300 (sm_103a) fused D2Q9 stream + collide + local kinetic sensor library.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/kss.h``); ``kss`` is its thin Python binding and ``inputs`` the seeded
synthetic workload generators.  Importing the package does not load the CUDA
library; ``kss.load()`` (or creating a ``kss.Lattice``) does, and raises if it is
missing.
"""

__all__ = ["kss", "inputs"]
