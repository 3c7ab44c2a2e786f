"""GB300 (sm_103a) CUDA kernels for sparse forward and reverse-mode automatic
differentiation of CSR operations (arXiv 2212.05159).

The compute lives in the in-tree CUDA library ``_build/libspx.so`` (C ABI in
``include/spx.h``); this package is its thin Python binding plus autograd glue.
"""
from . import abi, spai
from .csr import CSR
from .ops import SpAddPlan, SpGEMMPlan, TriangularSolver, masked_outer, sddmm, spadd, spgemm, spmm, spmm_t

__all__ = ["abi", "CSR", "spmm", "sddmm", "spmm_t", "masked_outer", "spgemm", "SpGEMMPlan", "spadd", "SpAddPlan", "TriangularSolver", "spai"]
