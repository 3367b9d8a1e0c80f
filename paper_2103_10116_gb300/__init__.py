"""GB300-native sparse SpMV and Krylov solvers (libspx).

The compute path is the CUDA library ``lib/libspx.so`` built from ``csrc/``
for sm_103a; ``spx`` is its thin ctypes binding (same names as the C ABI in
``include/spx.h``); ``synth`` draws seeded synthetic matrices.  Importing this
package does not load the CUDA library; ``spx.load()`` (called by every
binding function) does, and raises if it is missing.
"""
__all__ = ["spx", "synth", "build"]
