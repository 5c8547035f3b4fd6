"""GB300-native minimal-rank H^2 VIE matrix-vector product and Krylov solve.

The compute path is the CUDA C-ABI library libh2 (include/h2.h); `h2` is its
ctypes binding. `build.build_all()` compiles the native code in-tree.
"""
from .h2 import H2Arrays, H2Error, H2Matrix, arrays_from_blocks, lib  # noqa: F401
