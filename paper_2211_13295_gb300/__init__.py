"""GB300-native ADER-WENO zone update for the compressible Euler equations.

The compute path is the CUDA library ``libawe.so`` (built from ``csrc/`` by
``paper_2211_13295_gb300.build``) behind the C ABI declared in
``include/awe.h``; ``paper_2211_13295_gb300.awe`` is its ctypes binding.
``problems`` holds the seeded synthetic inputs.  Importing the package does
not load the CUDA library; creating a grid does, and fails loudly if the
library is missing.
"""
__all__ = ["problems", "awe"]
