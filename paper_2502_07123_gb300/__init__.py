"""GB300-native nested MLMC hot path (arXiv 2502.07123).

The compute path is the CUDA library ``libmlmc_gb300.so`` (C ABI declared in
include/mlmc.h); ``paper_2502_07123_gb300.mlmc`` is its thin Python binding.
"""
