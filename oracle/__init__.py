"""CPU oracle of RLOBPCG -- TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import this package. The GPU library shares no code with it and never
calls it; see ``oracle/rlobpcg.py`` for what it computes and how each piece is pinned.
"""
from .rlobpcg import *  # noqa: F401,F403
