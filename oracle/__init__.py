"""FP64 CPU oracle for entropic domain decomposition (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this package. The CUDA library shares no code with it.
"""
from .dd import *  # noqa: F401,F403
from . import dd, referees  # noqa: F401
