"""GB300-native time-stepper for the 3D Schroedinger equation closed by the
discrete Dirichlet-to-Neumann absorbing boundary condition (Wu & Li, Sec. 2-3).

The compute path is the native library ``_lib/libabc.so`` (CUDA kernels for
sm_103a plus an FP64 host setup), reached through ``paper_1908_02456_gb300.abc``.
Importing this package does not load the library; ``abc.load()`` does, and it
raises if the library is missing.
"""
__all__ = ["abc", "inputs"]
