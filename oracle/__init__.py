"""FP64 CPU oracle for hypothesis scoring (test infrastructure only).

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  The product path never calls it.
"""
from .oracle import *  # noqa: F401,F403
