"""GB300 (sm_103a) implementation of the damped real Chebyshev wave-packet hot path of
MADWAVE3 (arXiv 2412.10167): a C-ABI CUDA library (``libmw3.so``, built from ``csrc/``)
and its Python binding ``mw3``. Build with ``paper_2412_10167_gb300.build.build()``."""
