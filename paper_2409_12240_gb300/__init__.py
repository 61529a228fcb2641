"""GB300-native hot path of the graph tensor-network quantum annealer (arXiv:2409.12240).

The compute path is libgtqa.so (hand-written CUDA for sm_103a, C ABI in
include/gtqa.h); this package holds its build step and a thin ctypes binding.
"""
from . import gtqa  # noqa: F401
from ._build import build  # noqa: F401
