"""GB300-native Reed-Solomon erasure coding in the polynomial realization,
with the Vandermonde and Cauchy bit-matrix realizations as peers.

The compute path is the CUDA library ``librs_gb300.so`` (sm_103a kernels
behind a C ABI, declared in include/rs_gb300.h); ``paper_1312_5155_gb300.rs``
is its thin Python binding.  Importing this package does not load the
library; the binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "rs"]
