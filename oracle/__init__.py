"""FP64 CPU oracle for the P-APG iteration of Aybat & Wang (arXiv:1407.7220).

TEST INFRASTRUCTURE ONLY: the independent reference that the CUDA path is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
product package.
"""
from .oracle import *  # noqa: F401,F403
