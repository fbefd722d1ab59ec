"""dgsrhd: GB300-native nodal discontinuous-Galerkin special-relativistic hydrodynamics.

The hot path of arXiv 2205.00095 (conserved-to-primitive recovery, nodal DG right-hand side
with LLF/HLL fluxes, the physicality-enforcing operator, SSP-RK steps and the right-hand
side's vector-Jacobian product) runs in the CUDA library ``libdgsrhd.so`` behind the C ABI of
``include/dgsrhd.h``; this package builds it (``build``), binds it (``_lib``) and wraps it
for torch tensors (``Solver``)."""
from . import build
from ._lib import DGSRHDError
from .solver import Solver

__all__ = ["Solver", "DGSRHDError", "build"]
