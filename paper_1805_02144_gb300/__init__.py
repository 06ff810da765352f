"""GB300-native exponential Rosenbrock shallow-water path (arXiv:1805.02144).

The computation lives in the CUDA library ``libswe_exprb.so`` (C ABI in
``include/swe_exprb.h``); ``api`` is its Python binding with the same names,
``inputs`` generates seeded synthetic states and ``build`` compiles the
library for sm_103a.
"""

__all__ = ["api", "inputs", "build"]
