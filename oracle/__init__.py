"""FP64 CPU oracle for the MLCC3 triples path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The library itself never calls it, and it
shares no code with the CUDA path.
"""
from .mlcc3_oracle import *  # noqa: F401,F403
from .cnto import *  # noqa: F401,F403
