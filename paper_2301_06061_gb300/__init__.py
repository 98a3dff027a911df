"""GB300-native w-stacking imager (arXiv:2301.06061): gridding, per-plane 2D FFT and
w-correction phase screen as hand-written sm_103a CUDA kernels behind a C ABI.

``wst`` is the ctypes binding of ``libwst.so``; ``synth`` holds the seeded input
generators.  Importing the package does not load the CUDA library.
"""
__version__ = "0.1.0"
