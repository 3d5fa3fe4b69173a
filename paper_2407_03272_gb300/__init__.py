"""GB300-native accelerated Jacobi (AJ) solver for sparse SPSD systems.

The compute path is libaj (CUDA, sm_103a) behind the C ABI of include/aj.h;
``paper_2407_03272_gb300.aj`` is its ctypes binding.
"""
from . import aj  # noqa: F401
from .aj import Context, from_csr, lib, params, solve_batch  # noqa: F401
