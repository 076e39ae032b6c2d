"""GB300-native multi-Slater-determinant table method (Clark et al., arXiv:1106.2456).

Importing the package loads nothing heavy.  The CUDA path lives in the shared
library ``libmsd`` (C ABI declared in ``include/msd.h``); ``paper_1106_2456_gb300.msd``
is its thin Python binding and raises if the library or a GPU is missing.
"""
__all__ = ["workloads", "msd", "build"]
