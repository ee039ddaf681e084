"""GB300-native hierarchical 3D Gaussian splatting (RetinaGS, arXiv 2406.11836).

The compute path lives in the CUDA library under ``csrc/`` behind the C ABI declared in
``include/rgs.h``; ``rgs`` is its thin Python binding.  Importing this package loads
nothing; ``paper_2406_11836_gb300.rgs`` loads the library and fails loudly if it is
missing.
"""
__all__ = ["workloads"]
