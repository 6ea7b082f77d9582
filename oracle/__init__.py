"""FP64 CPU oracle for the PPPM k-space path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The product library never calls
it, links it or reads anything it writes, and the oracle imports nothing from
the product package.
"""
from .pppm_oracle import *  # noqa: F401,F403
from .ewald import *  # noqa: F401,F403
