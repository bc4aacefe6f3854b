"""GB300-native purified quantics-MPS Lindblad stepper.

The compute path is the C-ABI library ``libqlb.so`` (hand-written CUDA for
sm_103a, sources in ``csrc/``, declared in ``include/qlb.h``).  ``qlb`` is a thin
ctypes binding with the same call names.  ``inputs`` holds the seeded synthetic
workloads.  Importing this package does not load the library; ``qlb.load()``
does, and raises if it has not been built.
"""
