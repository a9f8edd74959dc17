"""GB300-native backward ray-shooting for gravitational microlensing (arXiv:1703.09707).

The compute lives in libmlens.so (CUDA for sm_103a, C ABI in include/mlens.h);
`paper_1703_09707_gb300.mlens` is its ctypes binding and `build` compiles it.
"""
from . import build  # noqa: F401

__all__ = ["build", "mlens"]
