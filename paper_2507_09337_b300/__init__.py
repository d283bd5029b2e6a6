"""B300-native block-hydro packet engine (arXiv 2507.09337, ORCHA's GPU task
function on a data packet of mesh blocks).

The compute path is the C-ABI library ``liborcha.so`` (CUDA kernels for
sm_103a, declared in ``include/orcha.h``); :mod:`.binding` is a thin ctypes
layer over it with the same names. Importing this package does not load the
library; :func:`binding.lib` does, and raises if it is missing.
"""
__all__ = ["workloads", "binding"]
