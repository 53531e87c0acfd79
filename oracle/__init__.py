"""FP64 CPU oracle for fast randomized singular value thresholding (FRSVT).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or helpers with the CUDA path in ``paper_1509_00296_gb300``; the
only thing both sides agree on is the published definition of the counter-based
Philox4x64-10 generator (Salmon et al., SC'11) that draws the Gaussian test
matrix Omega, which each side implements on its own.

Everything is computed in float64 with plain numpy / scipy primitives, written
to be checked against Oh, Matsushita, Tai and Kweon, "Fast Randomized Singular
Value Thresholding for Low-rank Optimization" (arXiv:1509.00296) by eye:

- ``philox``  : Philox4x64-10 and the Box-Muller map that produce Omega
                (Alg. 1 "Sample Gaussian random matrix"; Sec. 2.4).
- ``linalg``  : one-sided Jacobi SVD, cyclic Jacobi eigensolver, Newton polar
                decomposition (Def. 2, Sec. 2.2), QR with column pivoting
                (Sec. 2.1), modified Gram-Schmidt (range propagation, Sec. 2.1).
- ``svt``     : exact SVT (Def. 1, Eq. 3), FRSVT (Alg. 1, Eq. 6) with range
                propagation, weighted SVT, the 2-norm-ball projection (Def. 3).
- ``rpca``    : robust PCA by the inexact augmented Lagrange multiplier method
                that hosts the SVT (Sec. 4.1, "Robust PCA test").
- ``adjoint`` : the exact-SVD vector-Jacobian product of SVT.

Parity status of each function is stated in its module header.
"""
