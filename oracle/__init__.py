"""FP64 CPU oracle for coverage trajectory synthesis (arXiv 2511.11514).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  It shares no code with
the CUDA library (``paper_2511_11514_b300``) and neither imports the other.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, limits, library routines or brute force; the one exception is the
full outer loop ``solve``, pinned only through its parts and a one-iteration
composition check (see the header of ``oracle.py``).
"""
from .oracle import *  # noqa: F401,F403
