"""GB300-native direct kinematic scattering (Favre-Nicolin et al., J. Appl. Cryst. 2010).

The compute path is libscatter.so (CUDA, sm_103a) behind the C ABI declared in
include/scatter.h; this package holds its build script (``build``), a thin
ctypes binding with the same entry-point names (``binding``), a PyTorch
front end (``api``) and seeded input generators (``workloads``).  The CUDA
library is loaded on first use; a missing library raises immediately — there
is no CPU fallback.
"""
__all__ = ["build", "binding", "api", "workloads"]
