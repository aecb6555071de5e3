"""FP64 CPU oracle of the Gibbs TOD step.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import it.  It is independent of the CUDA
library (no shared code); see ``core`` for the definitions and citations.
"""
from .core import *  # noqa: F401,F403
from . import _huff  # noqa: F401
