"""FP64 CPU oracle of jackknife CP-ALS (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library never does.  See
``oracle/cp_als.py`` for what it computes and which passages it follows.
"""
from .cp_als import *  # noqa: F401,F403
from .cp_als import __all__  # noqa: F401
