"""Flowtree CPU oracle (test infrastructure only).

A plain FP64 restatement of the Flowtree estimate written from the paper
(arXiv 1910.04126, Sec. 2, Sec. 3, App. A.1, Eq. 1).  It shares no code with
the CUDA library.  Only the tests, the smoke check and the benchmark's CPU
baseline may import it; the library itself never does.
"""
from .oracle import *  # noqa: F401,F403
