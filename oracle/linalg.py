"""Dense FP64 factorizations used by the FRSVT oracle (test infrastructure only).

- ``jacobi_svd``   one-sided (Hestenes) Jacobi SVD with QR preconditioning.  It is
                   the oracle's SVD for the exact SVT of Def. 1 / Eq. 3.
                   Pinned against LAPACK (numpy.linalg.svd) and by invariants.
- ``jacobi_eig``   cyclic two-sided Jacobi eigensolver for symmetric matrices.
                   It is step 18 of Alg. 1 ([V, D] = EigenDecomposition(P)).
                   Pinned against LAPACK (numpy.linalg.eigh).
- ``newton_polar`` Newton iteration with Frobenius-norm scaling for the polar
                   decomposition C = W P (Def. 2; Sec. 2.2 cites Higham for it).
                   It is step 17 of Alg. 1.  Pinned against the SVD-based polar
                   factors.
- ``qr_cp``        QR with column pivoting and a rank cut (Sec. 2.1: the paper
                   uses LAPACK dgeqp3 + orgqr; here scipy's wrapper of the same
                   routine is the library primitive).
- ``mgs``          modified Gram-Schmidt orthogonalization of new columns
                   against an existing orthonormal block (range propagation,
                   Sec. 2.1 and Alg. 1 step 10).  Pinned by orthonormality and
                   span checks.

Sweeps of the Jacobi methods visit the disjoint index pairs of a round-robin
schedule, so that every rotation of a round can be applied at once with numpy;
each rotation is the textbook one.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def _round_robin(n: int):
    """Rounds of disjoint index pairs that together cover every pair (i < j) once."""
    N = n + (n % 2)
    players = list(range(N))
    rounds = []
    for _ in range(N - 1):
        ps, qs = [], []
        for k in range(N // 2):
            a, b = players[k], players[N - 1 - k]
            if a < n and b < n:
                ps.append(min(a, b))
                qs.append(max(a, b))
        if ps:
            rounds.append((np.array(ps), np.array(qs)))
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def _rotation_tangent(zeta: np.ndarray) -> np.ndarray:
    """Smaller root t of t^2 + 2 zeta t - 1 = 0 (the rotation angle of magnitude <= pi/4)."""
    sgn = np.where(zeta >= 0.0, 1.0, -1.0)
    return sgn / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))


def _one_sided_jacobi(X: np.ndarray, tol: float, max_sweeps: int):
    """Orthogonalize the columns of X (m x k) by plane rotations.

    Returns (Xr, R, sweeps) with X R = Xr, R orthogonal and the columns of Xr
    mutually orthogonal to relative accuracy tol.  Columns are held as the
    rows of one transposed array [X^T | R^T], so that each rotation updates
    the column of X and the column of R together on contiguous data.
    Columns whose squared norm is below (eps ||X||_F)^2 are not rotated: they
    cannot change any result by more than rounding.
    """
    m, k = X.shape
    T = np.hstack([np.array(X.T, dtype=np.float64), np.eye(k)])
    small = (np.finfo(np.float64).eps * np.linalg.norm(X)) ** 2
    rounds = _round_robin(k)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for p, q in rounds:
            tp, tq = T[p], T[q]
            gp, gq = tp[:, :m], tq[:, :m]
            alpha = np.einsum("ij,ij->i", gp, gp)
            beta = np.einsum("ij,ij->i", gq, gq)
            gamma = np.einsum("ij,ij->i", gp, gq)
            act = (np.abs(gamma) > tol * np.sqrt(alpha * beta)) & (alpha > small) & (beta > small)
            if not act.any():
                continue
            rotated = True
            zeta = (beta[act] - alpha[act]) / (2.0 * gamma[act])
            t = _rotation_tangent(zeta)
            c = (1.0 / np.sqrt(1.0 + t * t))[:, None]
            s = c * t[:, None]
            mp, mq = tp[act], tq[act]
            T[p[act]] = c * mp - s * mq
            T[q[act]] = s * mp + c * mq
        if not rotated:
            break
    return np.ascontiguousarray(T[:, :m].T), np.ascontiguousarray(T[:, m:].T), sweeps


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 80):
    """Thin SVD A = U diag(s) V^T by one-sided Jacobi; s is sorted in descending order.

    QR preconditioning (Drmac and Veselic): A P = Q R with column pivoting,
    then the columns of R^T are orthogonalized, R^T W = U_x Sigma, so that
    A = (Q W) Sigma (P U_x)^T.  A wide A is handled through A^T.
    Returns (U, s, Vt) with U: m x k, s: k, Vt: k x n, k = min(m, n).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        U, s, Vt = jacobi_svd(A.T, tol, max_sweeps)
        return Vt.T, s, U.T
    if n == 0:
        return np.zeros((m, 0)), np.zeros(0), np.zeros((0, n))
    Qp, R, piv = scipy.linalg.qr(A, mode="economic", pivoting=True)
    Xr, W, _ = _one_sided_jacobi(R.T, tol, max_sweeps)     # R^T W = Xr
    sig = np.sqrt(np.einsum("ij,ij->j", Xr, Xr))
    order = np.argsort(-sig, kind="stable")
    sig, Xr, W = sig[order], Xr[:, order], W[:, order]
    Ux = np.zeros_like(Xr)
    nz = sig > 0.0
    Ux[:, nz] = Xr[:, nz] / sig[nz]
    if not nz.all():
        # complete U_x with an orthonormal basis of the complement (zero singular values)
        k0 = int(nz.sum())
        Qc, _ = np.linalg.qr(np.hstack([Ux[:, :k0], np.eye(n)]))
        Ux[:, k0:] = Qc[:, k0:n]
    V = np.empty_like(Ux)
    V[piv, :] = Ux                              # P U_x
    return Qp @ W, sig, V.T


def jacobi_eig(S: np.ndarray, tol: float = 1e-15, max_sweeps: int = 80):
    """Symmetric eigendecomposition S = V diag(d) V^T by cyclic two-sided Jacobi.

    Eigenvalues are returned in descending order with matching columns of V.
    """
    S = np.array(S, dtype=np.float64)
    n = S.shape[0]
    S = 0.5 * (S + S.T)
    V = np.eye(n)
    if n <= 1:
        return np.diag(S).copy(), V
    rounds = _round_robin(n)
    scale = np.linalg.norm(S)
    if scale == 0.0:
        return np.zeros(n), V
    for _ in range(max_sweeps):
        rotated = False
        for p, q in rounds:
            spq = S[p, q]
            act = np.abs(spq) > tol * scale
            if not act.any():
                continue
            rotated = True
            p, q, spq = p[act], q[act], spq[act]
            theta = (S[q, q] - S[p, p]) / (2.0 * spq)
            t = _rotation_tangent(theta)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            J = np.eye(n)
            J[p, p] = c
            J[q, q] = c
            J[p, q] = s
            J[q, p] = -s
            S = J.T @ S @ J
            S = 0.5 * (S + S.T)
            V = V @ J
        if not rotated:
            break
    d = np.diag(S).copy()
    order = np.argsort(-d, kind="stable")
    return d[order], V[:, order]


def newton_polar(C: np.ndarray, tol: float = 1e-14, max_iter: int = 100):
    """Polar decomposition C = W P of a non-singular square C by scaled Newton iteration.

    X_{k+1} = (zeta_k X_k + X_k^{-T} / zeta_k) / 2 with the Frobenius-norm
    scaling zeta_k = sqrt(||X_k^{-1}||_F / ||X_k||_F); scaling is dropped once
    the iteration is in its quadratic regime.  W is the limit, P = W^T C
    (symmetrized).  Returns (W, P, iterations).
    """
    X = np.array(C, dtype=np.float64)
    if X.size == 0:
        return X.copy(), X.copy(), 0
    scaled = True
    it = 0
    for it in range(1, max_iter + 1):
        Xi = np.linalg.inv(X)
        zeta = np.sqrt(np.linalg.norm(Xi) / np.linalg.norm(X)) if scaled else 1.0
        Xn = 0.5 * (zeta * X + Xi.T / zeta)
        delta = np.linalg.norm(Xn - X) / np.linalg.norm(Xn)
        X = Xn
        if delta < 1e-2:
            scaled = False
        if delta <= tol:
            break
    W = X
    P = W.T @ C
    P = 0.5 * (P + P.T)
    return W, P, it


def qr_cp(Y: np.ndarray, rank_tol: float = 1e-12):
    """Orthonormal basis of range(Y) by QR with column pivoting and a rank cut.

    Keeps the leading s columns with |R_jj| > rank_tol * |R_00| (the pivoted
    diagonal is non-increasing), i.e. s = min(l, numerical rank).
    """
    Y = np.asarray(Y, dtype=np.float64)
    if Y.shape[1] == 0:
        return np.zeros((Y.shape[0], 0))
    Q, R, _ = scipy.linalg.qr(Y, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    if d.size == 0 or d[0] == 0.0:
        return np.zeros((Y.shape[0], 0))
    s = int(np.sum(d > rank_tol * d[0]))
    return np.ascontiguousarray(Q[:, :s])


def qr(Y: np.ndarray):
    """Thin Householder QR without pivoting (LAPACK through numpy)."""
    return np.linalg.qr(np.asarray(Y, dtype=np.float64))


def mgs(Qt: np.ndarray, Y: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """Modified Gram-Schmidt: orthonormalize the columns of Y against Qt and each other.

    Only the new columns are processed (the partial orthogonalization of range
    propagation); a column whose residual norm is <= rank_tol times its
    original norm is dropped.  Returns the accepted new orthonormal columns.
    """
    basis = [Qt[:, j] for j in range(Qt.shape[1])]
    out = []
    for j in range(Y.shape[1]):
        v = np.array(Y[:, j], dtype=np.float64)
        nrm0 = np.linalg.norm(v)
        for b in basis:
            v = v - (b @ v) * b
        nrm = np.linalg.norm(v)
        if nrm0 > 0.0 and nrm > rank_tol * nrm0:
            v = v / nrm
            basis.append(v)
            out.append(v)
    if not out:
        return np.zeros((Y.shape[0], 0))
    return np.stack(out, axis=1)
