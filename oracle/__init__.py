"""Oracle for the SPVAR + simulated-annealing hot path (Alg. 1, Alg. 2).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the CUDA library never uses it.
"""
from .oracle import *  # noqa: F401,F403
