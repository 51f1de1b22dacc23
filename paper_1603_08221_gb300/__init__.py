"""GB300-native two-species MRT lattice Boltzmann hot path (arXiv:1603.08221).

Modules (the CUDA library ``liblbm_mix.so`` does the computing; these marshal):
  binding      ctypes binding of include/lbm_mix.h (LbmMix, LbmSweep, LbmAdjoint)
  autograd     torch.autograd.Function over the library's adjoint
  diagnostics  CL(t), separation rate and dimensionless time from the records
  study        the paper's Table 1 run as one sweep
  workloads    seeded problem definitions (no method arithmetic)
  build        nvcc build of the library for sm_103a
"""
