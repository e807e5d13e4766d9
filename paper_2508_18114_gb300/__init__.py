"""GB300-native low-rank Lindblad integrator for transmon readout (sm_103a).

The compute path is the CUDA library ``liblr.so`` (C ABI in include/lr.h);
``lr`` is its ctypes binding. Build with ``python -m paper_2508_18114_gb300.build``.
"""
from .lr import LowRankBatch, LrError, load_library  # noqa: F401

__all__ = ["LowRankBatch", "LrError", "load_library"]
