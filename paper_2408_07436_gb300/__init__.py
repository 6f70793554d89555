"""GB300-native M2L field translation for the 3D Laplace kernel-independent FMM.

The compute lives in a C-ABI shared library (``libm2l_gb300.so``, built from ``csrc/`` for
sm_103a); ``m2l`` is its thin Python binding. Importing this package does not load the
library: ``from paper_2408_07436_gb300 import m2l`` does, and raises if it was not built.
``workloads`` draws the seeded synthetic inputs.
"""

__all__ = ["m2l", "workloads", "build"]
