"""GB300-native Line-DG (line-based discontinuous Galerkin) hot path.

The compute path lives in the C-ABI library ``libldg.so`` (CUDA kernels for
sm_103a plus host set-up code); :mod:`paper_1204_1533_gb300.ldg` is the thin
ctypes binding with the same entry-point names. :mod:`.inputs` produces
seeded synthetic meshes and states. Importing the package does not load the
library; the binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "ldg"]
