"""GB300-native collision resolution for dense rigid-sphere suspensions.

The hot path of "A Bifidelity Proximal Quasi-Newton Method for Dense Rigid
Body Suspension Collision Resolution": the per-time-step LCP
0 <= x perp D^T M D x + b >= 0, with a boundary-integral Stokes mobility M
solved by GMRES over O(N^2) stresslet sums, and the Mono-PQN / Bi-PQN solvers.
All arithmetic runs in the CUDA library ``liblcp_gb300.so`` behind the C ABI
of ``include/lcp_gb300.h``; this package only marshals arguments.
"""
from .lcp import *  # noqa: F401,F403
from .lcp import LcpError, config_for  # noqa: F401
