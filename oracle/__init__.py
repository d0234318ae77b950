"""FP64 CPU oracle for the Gaussian-splatting renderer (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The product library never calls it.
"""
from .oracle import *  # noqa: F401,F403
