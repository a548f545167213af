"""Matrix-free squared-exponential kernel products, their adjoint and the HMC
leapfrog step of determinant-free fully Bayesian GP regression, on GB300.

The compute path is libkmv.so (hand-written sm_103a CUDA behind the C ABI in
include/kmv.h); this package is its Python binding.  Importing the package
does not load the library; ``binding.lib()`` does, and fails loudly if it was
not built.
"""
from .binding import Kmv, KmvError, Points, default_handle, lib, PRECISIONS  # noqa: F401

__all__ = ["Kmv", "KmvError", "Points", "default_handle", "lib", "PRECISIONS"]
