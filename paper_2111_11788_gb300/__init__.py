"""GB300-native batched coupled MLMC sample solve (arXiv 2111.11788 hot path).

The compute path is libmlmc.so (CUDA, sm_103a) behind the C ABI of
include/mlmc.h; ``paper_2111_11788_gb300.mlmc`` is its ctypes binding.
"""
from . import mlmc  # noqa: F401
