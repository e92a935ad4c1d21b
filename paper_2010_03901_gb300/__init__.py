"""GB300 (sm_103a) implementation of the 2D Fourier Continuation hot path.

The compute library is ``_lib/libfc2d.so`` (C ABI in include/fc2d.h), built by
``paper_2010_03901_gb300.build.build()``; ``paper_2010_03901_gb300.fc2d`` is its
ctypes binding.  Importing this package does not load the library.
"""
