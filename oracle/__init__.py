"""CPU FP64 oracle for the POLFED hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The GPU
library never calls it and shares no code with it.
"""
from .polfed_oracle import *  # noqa: F401,F403
