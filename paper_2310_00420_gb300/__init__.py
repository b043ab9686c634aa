"""GB300-native covariance-free EM for clustered multi-task compressive sensing.

The compute path lives in ``libcmcs.so`` (CUDA for sm_103a, C ABI declared in
``include/cmcs.h``); ``cmcs`` is its thin ctypes binding and ``synth`` the seeded synthetic
workload generator.  Importing this package loads nothing native; the binding loads the
library on first use and raises if it is missing.
"""
