"""FP64 CPU oracle for arXiv:1206.3215 (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1206_3215_gb300`` never does, and the two share no code.
"""
from .oracle import *  # noqa: F401,F403
