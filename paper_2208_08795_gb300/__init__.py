"""GB300-native NPDU-AFPS (arXiv 2208.08795): the sampling hot path as CUDA
kernels for sm_103a behind a C ABI (``include/afps.h``).

The ctypes binding lives in :mod:`paper_2208_08795_gb300.afps` and is loaded
on first use, so that the input generators in :mod:`.synth` import without a
built library.
"""
