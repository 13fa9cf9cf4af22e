"""GB300-native fused-cluster state-vector simulator (Haener & Steiger, Sec. 2-3).

The compute path lives in libqs.so (include/qs.h); ``qs`` is its ctypes binding.
"""
from . import qs  # noqa: F401
