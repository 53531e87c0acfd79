"""GB300-native fast randomized singular value thresholding (FRSVT) and RPCA by inexact ALM.

The compute path is the C-ABI library ``libfrsvt.so`` (CUDA kernels for
sm_103a); ``paper_1509_00296_gb300.frsvt`` is its thin ctypes binding.  Importing
the package does not load the library; the first call that needs it does, and
raises if it has not been built.
"""
