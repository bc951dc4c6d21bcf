"""GB300 (sm_103a) implementation of the per-iteration hot path of the implicit
gas-kinetic scheme (Pan, Zhong & Zhuo, arXiv:1709.00803): CUDA kernels behind the C ABI
of include/igks.h, with a thin Python binding in `igks`."""
from . import igks  # noqa: F401

__all__ = ["igks"]
