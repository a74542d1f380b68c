"""GB300-native solver for sequences of Poisson problems: deflated PCG with Krylov
subspace recycling on the domain-decomposition interface problem, preconditioned
by two-/three-level BDDC (arXiv 2412.17543).

The numerical work runs in the native library libdd_gb300.so (hand-written sm_103a
CUDA kernels behind the C ABI of include/dd_solver.h); this package is its thin
binding. Build it with `python -m paper_2412_17543_gb300.build` or
`__graft_entry__.build()`.
"""
from .api import PoissonSolve, Recycler, Solver, make_options, plan  # noqa: F401
from ._native import DDError, load  # noqa: F401
