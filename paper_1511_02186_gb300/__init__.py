"""GB300-native Adaptive Inverse Distance Weighting (Mei, Xu & Xu, arXiv 1511.02186).

The hot path lives in ``libaidw.so`` (hand-written CUDA for sm_103a behind the C ABI of
``include/aidw.h``); ``aidw`` is its Python binding (the library is loaded on first use) and
``workloads`` the seeded synthetic inputs.
"""
from . import aidw, workloads  # noqa: F401
