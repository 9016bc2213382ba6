"""FP64 CPU oracle for the EFGP hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library never does.
"""
from .efgp_oracle import *  # noqa: F401,F403
from .efgp_oracle import Kernel, OracleResult, efgp  # noqa: F401
