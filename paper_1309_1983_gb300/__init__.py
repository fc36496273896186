"""GB300-native D3Q19 BGK lattice Boltzmann hot path (Mawson & Revell,
"Memory transfer optimization for a lattice Boltzmann solver on Kepler
architecture nVidia GPUs").

The compute runs in hand-written CUDA kernels for sm_103a behind the C-ABI
library ``liblbm.so`` (declared in ``include/lbm.h``); this package is the
thin Python binding over it. Importing the package does not load the
library: the first use of :mod:`paper_1309_1983_gb300.capi` does, and fails
loudly if it has not been built.
"""

__all__ = ["capi", "lattice", "workloads"]
