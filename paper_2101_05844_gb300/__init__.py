"""GB300 (sm_103a) implementation of the batched hot path of the sparse dual solvers of
De Palma et al., "Scaling the Convex Barrier with Sparse Dual Algorithms" (arXiv 2101.05844).

  synth    seeded synthetic workloads (no method arithmetic)
  binding  ctypes binding of the C ABI (include/convex_barrier.h); the CUDA library is
           libconvex_barrier.so in this directory, built by build.py
  autograd torch.autograd.Function over the bound and its envelope gradient
"""
