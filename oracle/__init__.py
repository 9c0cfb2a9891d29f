"""CPU oracle for the block COCG / block COCR iterations (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library never calls it and shares no code with it.
"""
from .blcoc_oracle import *  # noqa: F401,F403
