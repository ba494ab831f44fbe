"""GB300-native jackknife CP-ALS (JK-CALS): the concurrent jackknife MTTKRP and
the per-submodel Gram-Hadamard / Cholesky / normalise / fit kernels behind it.

The compute path is the C-ABI library ``libjkcals.so`` (hand-written sm_103a
CUDA); this package is its thin Python binding.  There is no CPU fallback:
every call fails loudly when the library is missing.
"""
