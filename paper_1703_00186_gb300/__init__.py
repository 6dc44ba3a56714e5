"""GB300-native D2Q37 thermal lattice Boltzmann step (sm_103a CUDA kernels behind a C ABI).

Modules:
  _lib     ctypes binding of liblbm.so (include/lbm.h)
  lbm      Lattice: one lattice in HBM (init, step, moments, adjoint step)
  adjoint  checkpointed adjoint rollouts as a torch.autograd.Function
  batch    many independent lattices stepped by one CUDA graph
  build    in-tree build of liblbm.so
"""
__all__ = ["lbm", "adjoint", "batch", "build"]
