"""GB300-native HDG static-condensation library (arXiv 1807.00086, Sec. 2.4).

The compute path is the CUDA shared library ``libhdg.so`` built from ``csrc/`` for
sm_103a; ``hdg`` (the ctypes binding) only marshals arguments. Importing this package
does not load the library; ``paper_1807_00086_gb300.hdg`` does, and raises if the
library is missing.
"""
