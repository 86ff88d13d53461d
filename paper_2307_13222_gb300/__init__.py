"""GB300 (sm_103a) library for the matrix-free H*x of spin-1/2 and Hubbard
models and the Lanczos / canonical-TPQ drivers built on it (arXiv 2307.13222).

The product is the C-ABI shared library described by include/hphi.h (CUDA
sources in csrc/, built by build.py); `hphi` is its thin Python binding.
"""
from .build import build, LIB as LIBRARY_PATH
from . import hphi
from .hphi import (Context, Basis, Hamiltonian, HphiError, hphi_apply_H, hphi_dot, hphi_nrm2, hphi_axpy, hphi_scal,
                   hphi_random_vector, hphi_lanczos, hphi_tpq_step, hphi_dump_pattern, hphi_tridiag_eigen,
                   write_matrix_market, load_library)

__all__ = ["build", "LIBRARY_PATH", "hphi", "Context", "Basis", "Hamiltonian", "HphiError", "hphi_apply_H",
           "hphi_dot", "hphi_nrm2", "hphi_axpy", "hphi_scal", "hphi_random_vector", "hphi_lanczos",
           "hphi_tpq_step", "hphi_dump_pattern", "hphi_tridiag_eigen", "write_matrix_market", "load_library"]
