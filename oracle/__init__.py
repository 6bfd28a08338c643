"""FP64 CPU oracle for the proximal distance convex-clustering algorithm.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import it.  It shares no code with the
CUDA library (paper_1409_2065_gb300).
"""
from .pd_oracle import *  # noqa: F401,F403
