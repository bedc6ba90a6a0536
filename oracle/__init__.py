"""FP64 CPU oracle of the TDA-BSE hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import this package.  The product path (the C-ABI library and its
Python binding) never imports, links or runs anything here, and this package imports
nothing from the product path.
"""
from .bse_oracle import *  # noqa: F401,F403
