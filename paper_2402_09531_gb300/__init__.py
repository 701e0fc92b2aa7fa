"""GB300 (sm_103a) dimension-weighted fast multipole method.

The numerical path lives in libdwfmm.so (C ABI: include/dwfmm.h), built
in-tree by ``paper_2402_09531_gb300.build.build()``.  ``dwfmm`` is its thin
ctypes binding.
"""
from .dwfmm import (Batch, DwfmmError, Plan, EXPORTS, KERNELS, PRECISIONS, WEIGHT_RULES,  # noqa: F401
                    LIB_PATH, lib, load)

__all__ = ["Batch", "DwfmmError", "Plan", "EXPORTS", "KERNELS", "PRECISIONS", "WEIGHT_RULES",
           "LIB_PATH", "lib", "load"]
