"""CPU oracle of the Flow Fields patch-matching loop (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library under ``paper_1703_02563_gb300``
never does.
"""
from .ffo import *  # noqa: F401,F403
