"""CPU FP64 oracle for the compactly supported RBF least-squares surface fit.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute it.  It
shares no code with the CUDA library (no kernels, headers, helpers or tables).
"""
from .rbf_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401
from . import poly_oracle  # noqa: F401
from . import window_oracle  # noqa: F401
