"""GB300 (sm_103a) implementation of the Strang-split semi-Lagrangian
discontinuous Galerkin Vlasov-Poisson step of Einkemmer (arXiv 1803.02143).

The computation lives in ``libsldg.so`` (CUDA kernels behind the C ABI of
``include/sldg.h``); this package holds its ctypes binding (``_native``),
a PyTorch-memory front end (``solver``), the adjoint as a
``torch.autograd.Function`` (``autograd``) and the workload presets
(``configs``).
"""
from . import _native
from ._native import SldgError
from .solver import Config, Sldg

__all__ = ["Config", "Sldg", "SldgError", "_native"]
