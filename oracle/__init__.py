"""FP64 CPU oracle of the VP-LBM method (arXiv 2110.00967).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline
leg of the benchmark load it; the CUDA library never does.
"""
from .oracle import *  # noqa: F401,F403
