"""FP64 CPU oracle for the ISDF-SMW inverse dielectric matrix (test infrastructure).

This package is test infrastructure only: the tests, the smoke check and the
CPU-baseline leg of the benchmark call it; the library never does.  It
shares no code with the CUDA path.  See `oracle.isdf_oracle` for the
functions and the paper passages each one follows.
"""
from .isdf_oracle import *  # noqa: F401,F403
