"""GB300-native (sm_103a) implementation of the per-timestep hot path of the DPSNN
cortical simulator (Pastorelli et al., PDP 2018): LIF+SFA point neurons on a 2-D
grid of cortical modules, Gaussian or exponential lateral connectivity, integer
axonal delays.

The compute path is the C-ABI library ``libsnn.so`` (CUDA kernels for sm_103a);
``snn`` is its thin ctypes binding.  Importing this package loads nothing; the
library is loaded on first use and fails loudly when it is missing.
"""
__all__ = ["snn", "workloads"]
