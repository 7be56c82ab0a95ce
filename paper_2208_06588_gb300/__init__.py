"""GB300-native (sm_103a, FP64) solver for the 1D well-balanced ALE-WENO hybrid scheme.

The compute path is a CUDA shared library (``csrc/``) behind a C ABI (``include/swale.h``);
``binding`` marshals arguments to it through ctypes. Importing this package does not load the
library; the first binding call does, and it raises if the library is missing.
"""
