"""GB300 (sm_103a) solver for convex clustering by the proximal distance algorithm.

The solver is the CUDA library ``_lib/libccx.so`` behind the C ABI in
``include/ccx.h``; ``binding`` is its thin Python marshalling layer.
"""
from .binding import *  # noqa: F401,F403
from .binding import CcxError, GammaStats, KnnRule, Opts, Problem  # noqa: F401
