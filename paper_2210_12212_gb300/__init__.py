"""GB300-native IHS-BIN ridge-regularization-path library (C ABI + ctypes binding).

The compute path is the in-tree CUDA library ``libihsbin.so`` (built by
``paper_2210_12212_gb300.build``); :mod:`paper_2210_12212_gb300.ihsbin` is its
argument-marshalling binding.  Importing the package does not load the
library; ``ihsbin.load()`` does, and fails loudly if it is missing.
"""
