import os
import sys

# the oracle's sparse LU runs single-threaded (SuperLU); threaded BLAS under it
# only oversubscribes the cores (a 3,000-point factorisation went from 0.9 s to
# 75 s on a loaded host), so the test processes keep BLAS to one thread
for _k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_k, "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
