"""GB300-native random-batch list (RBL) short-range MD force step (arXiv 2105.04884).

The compute path is the CUDA library ``librbl`` (``csrc/``), reached through the
C-ABI declared in ``include/rbl.h``; ``paper_2105_04884_gb300.rbl`` is a thin ctypes
binding over it.  Importing this package loads nothing: ``rbl`` loads the library on
first use and raises if it has not been built.
"""
