"""GB300-native multilevel proximal-Newton solver for sparse inverse covariance.

The solver lives in a CUDA shared library behind a C ABI (include/glasso.h);
`paper_1607_00315_gb300.glasso` is the thin ctypes binding over it.  Importing
this package does not load the library; `glasso.load()` does, and fails
loudly when the library is missing.
"""
