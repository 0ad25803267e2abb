"""FP64 CPU oracle for the unaligned kernel-mode CP-HIFI subproblem.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may call it.  It shares no code with the CUDA path.
"""
from .cphifi_oracle import *  # noqa: F401,F403
from . import als_oracle  # noqa: F401  (the alternating fit around the kernel-mode solve)
