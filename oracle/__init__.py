"""CPU oracle (test infrastructure): plain SciPy sparse-LU NEGF transmission.

Only tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA path.
"""
from .negf_oracle import *  # noqa: F401,F403
