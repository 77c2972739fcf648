"""GB300-native RNS-CKKS homomorphic matrix multiplication (arXiv 2305.17341).

The compute path lives in libhe_gb300.so (hand-written CUDA for sm_103a,
sources in csrc/, C ABI in include/he.h).  This package is its thin ctypes
binding plus the build step; it has no CPU fallback.
"""
from . import _lib
from ._lib import *  # noqa: F401,F403
from .builder import build  # noqa: F401
