"""FP64 CPU oracle of the interior-penalty DG method (arXiv:1502.02941).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the product library.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
