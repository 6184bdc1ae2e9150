"""Sequential FP64 reference sampler -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product library never does.
"""
from .oracle import *  # noqa: F401,F403
