"""GB300 (sm_103a) library for PackVFL's encrypted MatMult (arXiv 2405.00482).

The compute path is the CUDA library libhe.so (C ABI in include/he.h); `he` is its
Python binding.  Importing this package loads nothing: `he` loads libhe.so on first use
and raises if it has not been built.
"""
