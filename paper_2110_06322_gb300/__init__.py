"""GB300 (sm_103a) closest point method solver: the hot path of arXiv 2110.06322.

Modules (imported explicitly; nothing here loads the CUDA library):
  cpm          ctypes binding of libcpm (include/cpm.h): Band, Schwarz, solve, solve_batch, ...
  autograd     differentiable solves and the checkpointed Schnakenberg integrator
  inputs       seeded synthetic inputs and the named workloads
  build        in-tree nvcc build of libcpm.so
(The measurement and profiling drivers are modes of bench.py at the repository root.)
"""
