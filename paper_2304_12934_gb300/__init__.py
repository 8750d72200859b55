"""GB300-native NUFFT Radon projector, back-projector and MBIR (tomoCAM, arXiv 2304.12934).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``); ``api`` is a thin ctypes binding over it.  Importing this package
loads nothing: the library is loaded on first use by ``api`` and raises if it
is missing.  ``synth`` draws seeded inputs only.
"""
__version__ = "0.1.0"
