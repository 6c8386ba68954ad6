"""GB300-native real-space NEGF transmission (absorbing boundary conditions).

The compute path lives in a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``), reached from Python through :mod:`.binding`.  Importing
this package loads nothing; ``binding.load()`` loads the library and raises if
it is missing.
"""
__version__ = "0.1.0"
