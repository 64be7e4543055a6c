"""B300-native (sm_103a) coupled TSLB + conservative Allen-Cahn step (arXiv 2501.00846).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI declared in
``include/lbm.h``; ``solver.py`` is a thin ctypes binding over it.  Importing this package does
not load the library; ``Solver`` does, and raises if it is missing.
"""
