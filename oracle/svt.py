"""Singular value thresholding operators in FP64 (test infrastructure only).

- ``exact_svt``      Def. 1 / Eq. 3: S_tau(A) = U S_tau(Sigma) V^T, with the
                     oracle's own one-sided Jacobi SVD.  Pinned by brute-force
                     minimization of Eq. 2 on 4x3 inputs, diagonal and
                     orthogonally-invariant closed forms, the prox optimality
                     condition, and rank(X) = #{sigma_i > tau}.
- ``ball_projection``Def. 3: P_tau(A) = U min(Sigma, tau) V^T (A = S_tau(A) + P_tau(A)).
- ``frsvt``          Alg. 1 (FRSVT) step by step, with range propagation
                     (Sec. 2.1) and the polar + eigen route of Sec. 2.2 / Eq. 6.
                     Pinned by: equality with exact_svt when rank(A) <= l
                     (Sec. 3.1, remark after Cor. 2), invariance to the choice
                     of orthonormalization (Prop. 1), the Theorem 3 average
                     bound over Omega draws.  Under range propagation it reports
                     the residual norm ||(I - Q~ Q~^T) A^T omega|| of the first new
                     sample column (``extra["rp_residual"]``).
- ``residual_estimate`` Prop. 4 / Eq. 14: alpha sqrt(2/pi) ||(I - Q Q^T) y||.  Pinned
                     by the exact failure rate of the bound for a rank-one residual
                     (|g| < 1 / (alpha sqrt(2/pi)), g ~ N(0, 1)), the mean of the
                     residual norm (sqrt(2/pi) sigma), the 1 - 1/alpha guarantee and
                     the zero residual when Q spans the range.
- ``wsvt``           weighted SVT (the WSVT footnote of Sec. 1): U max(Sigma - w, 0) V^T.
                     Pinned by reduction to SVT for constant weights and by
                     brute-force minimization of the weighted problem on 4x3
                     inputs with non-descending weights.
- ``wnnm_weights``   the WNNM weight rule w_j = c sqrt(n) / (sigma_j + eps) of the
                     patch-group workload (weights from the input's own sigma_j).
- ``frsvt`` with ``weights``: Alg. 1 with the soft threshold of step 19 replaced
                     by the weighted one, max(D - w(D), 0), w evaluated on the
                     approximate singular values D.  Pinned by equality with
                     ``wsvt`` when rank(A) <= l and with the unweighted ``frsvt``
                     for constant weights.
- ``svt_vjp``        adjoint of the exact SVT (divided-difference form of the derivative
                     of a spectral function, and the tau derivative).  Pinned by central
                     finite differences of ``exact_svt`` in FP64.
- ``frsvt_vjp``      adjoint of the FRSVT map with a fixed Omega (Alg. 1 run backwards: the
                     SVT adjoint of the small problem, the QR adjoint of every
                     orthonormalisation, the transposed products).  Pinned by entrywise
                     central differences of ``frsvt`` (every entry of A and tau, tall and
                     wide inputs, q = 0..2) and by equality with ``svt_vjp`` when the basis
                     spans the short side (l = min(m, n): FRSVT is then the exact SVT).
- ``psvt``           partial SVT of the truncated nuclear norm (Table 6, Type B):
                     the k leading singular values are kept, the rest shrunk.

Readings of the paper used here (the paper is silent or self-contradictory):
- Orientation: the basis Q is put on the shorter side of A (Sec. 2.5 asks for
  m < n "by transposing"; footnote 2 assumes m >= n).  Omega therefore has
  max(m, n) rows, indexed by the long-side index.  A square A is treated like
  a tall one (the problem is transposed, Q lives on the column side).
- Rank cut of QR-CP: keep |R_jj| > rank_tol * |R_00|, rank_tol = 1e-12.
- Range propagation with a fixed l: keep Q~ = (QV)[:, :min(r, l - 2)] (the
  a = 2 floor of Eq. 7) and draw l - |Q~| new Gaussian columns; with an empty
  Q~ the plain sketch of l columns is used.
- r = #{sigma_i > tau} with a strict inequality; singular values equal to tau
  shrink to zero either way.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import linalg
from .philox import gaussian_matrix


def soft(x, tau):
    """Soft shrinkage S_tau(x) = sgn(x) max(|x| - tau, 0) (Def. 1)."""
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0)


def residual_norm(Q: np.ndarray, y: np.ndarray) -> float:
    """||(I - Q Q^T) y||_2 for an orthonormal Q (the Gram-Schmidt residual of Prop. 4)."""
    Q = np.asarray(Q, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.linalg.norm(y - Q @ (Q.T @ y)))


def residual_estimate(Q: np.ndarray, y: np.ndarray, alpha: float = 20.0) -> float:
    """Prop. 4 / Eq. 14: varsigma = alpha sqrt(2 / pi) ||(I - Q Q^T) A omega||_2 with y = A omega.

    With probability at least 1 - 1 / alpha over the Gaussian omega it bounds
    ||(I - Q Q^T) A||_2, hence sigma_{k+1}(A) for a rank-k Q (Lemma 3 with one draw).
    """
    return float(alpha * np.sqrt(2.0 / np.pi) * residual_norm(Q, y))


def exact_svt(A: np.ndarray, tau: float):
    """Exact SVT of Def. 1 (Eq. 3).  Returns (X, r) with r = #{sigma_i > tau}."""
    U, s, Vt = linalg.jacobi_svd(A)
    f = soft(s, tau)
    return (U * f) @ Vt, int(np.sum(s > tau))


def ball_projection(A: np.ndarray, tau: float) -> np.ndarray:
    """2-norm-ball Euclidean projection P_tau(A) = U min(Sigma, tau) V^T (Def. 3)."""
    U, s, Vt = linalg.jacobi_svd(A)
    return (U * np.minimum(s, tau)) @ Vt


def wsvt(A: np.ndarray, w: np.ndarray):
    """Weighted SVT: U diag(max(sigma_j - w_j, 0)) V^T for weights w (one per sigma_j).

    A callable w is evaluated on the singular values of A (e.g. the WNNM
    weights c * sqrt(n) / (sigma_j + eps)).
    """
    U, s, Vt = linalg.jacobi_svd(A)
    wv = w(s) if callable(w) else np.asarray(w, dtype=np.float64)
    f = np.maximum(s - wv, 0.0)
    return (U * f) @ Vt


def wnnm_weights(n: int, c: float, eps: float):
    """Weight rule of the WNNM patch groups: w_j = c sqrt(n) / (sigma_j + eps), n = columns."""
    return lambda sig: c * np.sqrt(float(n)) / (np.asarray(sig, dtype=np.float64) + eps)


def psvt(A: np.ndarray, tau: float, k: int):
    """Partial SVT for the truncated nuclear norm sum_{i>k} sigma_i (Table 6, Type B)."""
    U, s, Vt = linalg.jacobi_svd(A)
    f = s.copy()
    f[k:] = np.maximum(s[k:] - tau, 0.0)
    return (U * f) @ Vt


@dataclass
class FRSVTResult:
    """Output of one FRSVT call (Alg. 1 outputs plus diagnostics)."""

    X: np.ndarray                 # S_tau(A) approximation, m x n
    Q_tilde: np.ndarray           # propagated basis (QV)[:, :keep] on the short side
    r: int                        # #{sigma_i > tau}
    sigma: np.ndarray             # D of Alg. 1 (singular values of B), descending
    s: int                        # number of basis columns actually used
    polar_iters: int = 0
    extra: dict = field(default_factory=dict)


def frsvt(A: np.ndarray, tau: float, l: int, q: int, seed: int, stream: int,
          Q_prev: np.ndarray | None = None, rank_tol: float = 1e-12,
          problem: int = 0, weights=None, partial_k: int = 0, orth_last: bool = False) -> FRSVTResult:
    """Fast randomized SVT, Alg. 1, on A (m x n) in FP64.

    Omega is the (seed, stream, problem) Philox Gaussian matrix with max(m, n)
    rows; under range propagation (Q_prev given and non-empty) only its first
    p = l - |Q_prev| columns are used.  Q_prev lives on the short side of A.
    With ``weights`` (a callable on the singular values D of B), step 19
    shrinks by max(D - weights(D), 0) instead of S_tau(D) and r counts
    D_j > w_j.  With ``partial_k`` > 0 step 19 is the partial thresholding of
    the truncated nuclear norm (Table 6, Type B): the partial_k leading values
    of D are kept, the others soft-thresholded; r counts the non-zero ones.
    With ``orth_last`` the power iteration orthonormalises only after its last
    step (Sec. 2.5, Table 2 line 4): the intermediate steps carry A A^T Q on
    as it is.  The span, hence X, is the same in exact arithmetic.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    transposed = m >= n
    Ah = A.T if transposed else A          # short x long ("m < n" of Sec. 2.5); ties transpose
    ns, nl = Ah.shape
    if ns == 0 or nl == 0:
        return FRSVTResult(np.zeros_like(A), np.zeros((ns, 0)), 0, np.zeros(0), 0)
    l = min(l, ns)

    # Alg. 1 steps 3-12: sketch, with or without range propagation.
    rp_residual = -1.0                     # no propagated basis: Prop. 4 estimate unavailable
    if Q_prev is None or Q_prev.shape[1] == 0:
        Omega = gaussian_matrix(nl, l, seed, stream, problem)       # step 4
        Y = Ah @ Omega                                              # step 5
        Q = linalg.qr_cp(Y, rank_tol)                               # step 6
    else:
        p = l - Q_prev.shape[1]
        Omega = gaussian_matrix(nl, p, seed, stream, problem)       # step 8
        Y = Ah @ Omega                                              # step 9
        QY = linalg.mgs(Q_prev, Y, rank_tol)                        # step 10
        Q = np.hstack([Q_prev, QY])                                 # step 11
        # Prop. 4: the residual of the first new sample column against the propagated basis
        rp_residual = residual_norm(Q_prev, Y[:, 0]) if p > 0 else -1.0

    # Steps 13-15: power iteration Q = QR(A A^T Q), eta = q times.  The rank is
    # re-checked with a pivoted QR (Sec. 2.1, range propagation paragraph).
    for it in range(q):
        Y = Ah @ (Ah.T @ Q)
        Q = Y if (orth_last and it < q - 1) else linalg.qr_cp(Y, rank_tol)

    s = Q.shape[1]
    if s == 0:
        return FRSVTResult(np.zeros_like(A), np.zeros((ns, 0)), 0, np.zeros(0), 0)

    # Step 16: [H, C] = QR(A^T Q).
    H, C = linalg.qr(Ah.T @ Q)
    # Step 17: C = W P (Newton polar).  Step 18: P = V D V^T.
    W, P, pit = linalg.newton_polar(C)
    D, V = linalg.jacobi_eig(P)
    # Step 19 / Eq. 6: S_tau(A) ~= (QV) S_tau(D) (HWV)^T.
    QV = Q @ V
    HWV = H @ (W @ V)
    if weights is None:
        fD = soft(D, tau)
        if partial_k > 0:                          # partial thresholding (Table 6, Type B)
            fD[:partial_k] = D[:partial_k]
        r = int(np.sum(fD > 0.0)) if partial_k > 0 else int(np.sum(D > tau))
    else:
        wD = weights(D)
        fD = np.maximum(D - wD, 0.0)
        r = int(np.sum(D > wD))
    Xh = (QV * fD) @ HWV.T
    keep = min(r, l - 2)
    Q_tilde = np.ascontiguousarray(QV[:, :max(keep, 0)])          # step 21
    X = Xh.T if transposed else Xh
    return FRSVTResult(np.ascontiguousarray(X), Q_tilde, r, D, s, pit,
                       extra={"QV": QV, "rp_residual": rp_residual})


def wsvt_batch(mats, c: float, eps: float, variant: str = "exact", l: int = 12, q: int = 1,
               seed: int = 0, stream: int = 0):
    """Weighted SVT of each patch group with the WNNM weights of its own n_i.

    variant "exact": ``wsvt`` with weights from the exact sigma_j; "frsvt": Alg. 1 on the
    problem with Philox problem index b (its position in the batch) and the weights on D.
    """
    out = []
    for b, A in enumerate(mats):
        n = A.shape[1]
        w = wnnm_weights(n, c, eps)
        if variant == "exact":
            out.append(wsvt(A, w))
        else:
            out.append(frsvt(A, 0.0, l, q, seed, stream, problem=b, weights=w).X)
    return out


def svt_vjp(A: np.ndarray, tau: float, Xbar: np.ndarray):
    """Adjoint of the exact SVT X = S_tau(A) (Def. 1): returns (Abar, taubar) for the cotangent Xbar.

    With A = U diag(sigma) V^T (thin, k = min(m, n)), f_i = max(sigma_i - tau, 0) and
    Ubar = U^T Xbar V, the divided-difference form of the derivative of a spectral function:
        Abar = U K V^T + (I - U U^T) Xbar V diag(f / sigma) + U diag(f / sigma) U^T Xbar (I - V V^T),
        K_ij = Gs_ij sym(Ubar)_ij + Gk_ij skew(Ubar)_ij (i != j),  K_ii = f'(sigma_i) Ubar_ii,
        Gs_ij = (f_i - f_j) / (sigma_i - sigma_j)  (f' where the two coincide),
        Gk_ij = (f_i + f_j) / (sigma_i + sigma_j),
    and taubar = -sum_{sigma_i > tau} Ubar_ii (df_i / dtau = -1 above the threshold).
    """
    A = np.asarray(A, dtype=np.float64)
    Xbar = np.asarray(Xbar, dtype=np.float64)
    U, s, Vt = linalg.jacobi_svd(A)
    V = Vt.T
    f = np.maximum(s - tau, 0.0)
    fp = (s > tau).astype(np.float64)
    Ub = U.T @ Xbar @ V
    sym = 0.5 * (Ub + Ub.T)
    skw = 0.5 * (Ub - Ub.T)
    k = s.size
    Gs = np.empty((k, k))
    Gk = np.zeros((k, k))
    for i in range(k):
        for j in range(k):
            d = s[i] - s[j]
            Gs[i, j] = (f[i] - f[j]) / d if abs(d) > 1e-12 * max(s[0], 1e-300) else 0.5 * (fp[i] + fp[j])
            if s[i] + s[j] > 0:
                Gk[i, j] = (f[i] + f[j]) / (s[i] + s[j])
    K = Gs * sym + Gk * skw
    K[np.diag_indices(k)] = fp * np.diag(Ub)
    D = np.where(s > 0, f / np.where(s > 0, s, 1.0), 0.0)
    Abar = U @ K @ V.T
    Abar += (Xbar @ V - U @ (U.T @ Xbar @ V)) * D[None, :] @ V.T
    Abar += U @ (D[:, None] * (U.T @ Xbar - (U.T @ Xbar @ V) @ V.T))
    taubar = -float(np.sum(np.diag(Ub)[s > tau]))
    return Abar, taubar


def _qr_pos(Y: np.ndarray):
    """Thin QR with a non-negative diagonal of R (the unique factor of a full-rank Y)."""
    Q, R = linalg.qr(Y)
    sg = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * sg[None, :], R * sg[:, None]


def _qr_vjp(Q: np.ndarray, R: np.ndarray, Qbar: np.ndarray) -> np.ndarray:
    """Adjoint of the thin QR Y = Q R (full column rank) for a cotangent of Q alone.

    With M = -Qbar^T Q (the R R-bar^T term is absent: R feeds nothing downstream) and
    copyltu(M) = tril(M) + tril(M, -1)^T, Ybar = (Qbar + Q copyltu(M)) R^{-T}.
    """
    M = -(Qbar.T @ Q)
    C = np.tril(M) + np.tril(M, -1).T
    return np.linalg.solve(R, (Qbar + Q @ C).T).T


def frsvt_vjp(A: np.ndarray, tau: float, l: int, q: int, seed: int, stream: int, Xbar: np.ndarray,
              problem: int = 0):
    """Vector-Jacobian product of the FRSVT map with a fixed Omega (Alg. 1, no range propagation).

    Returns (Abar, taubar, X) for the cotangent Xbar of X = FRSVT_tau(A).  The forward is Alg. 1
    in the orientation of ``frsvt`` (Ah = the short x long view of A), with every
    orthonormalisation a thin QR (X depends only on the spans, Prop. 1, so this is the map
    ``frsvt`` computes with pivoted QR wherever no column is dropped):
        Y_0 = Ah Omega,  Q_0 R_0 = Y_0                              (steps 4-6)
        Z_i = Ah^T Q_{i-1},  Y_i = Ah Z_i,  Q_i R_i = Y_i, i = 1..q   (steps 13-15)
        B = Q_q^T Ah,  Xh = Q_q S_tau(B)                             (steps 16-19, Eq. 6)
    and the reverse pass takes the same steps backwards: the exact SVT adjoint of the small
    problem (``svt_vjp`` on B, divided differences), the QR adjoint of each factorisation
    (``_qr_vjp``), and the products' transposes.
    """
    A = np.asarray(A, dtype=np.float64)
    Xbar = np.asarray(Xbar, dtype=np.float64)
    m, n = A.shape
    transposed = m >= n
    Ah = A.T if transposed else A
    Xbh = Xbar.T if transposed else Xbar
    ns, nl = Ah.shape
    l = min(l, ns)
    Omega = gaussian_matrix(nl, l, seed, stream, problem)
    # forward, keeping what the reverse pass reads
    Qs, Rs, Zs = [], [], []
    Q, R = _qr_pos(Ah @ Omega)
    Qs.append(Q)
    Rs.append(R)
    for _ in range(q):
        Z = Ah.T @ Q
        Q, R = _qr_pos(Ah @ Z)
        Zs.append(Z)
        Qs.append(Q)
        Rs.append(R)
    B = Q.T @ Ah
    W, _ = exact_svt(B, tau)
    Xh = Q @ W
    # reverse
    Qbar = Xbh @ W.T                                  # Xh = Q W
    Wbar = Q.T @ Xbh
    Bbar, taubar = svt_vjp(B, tau, Wbar)              # W = S_tau(B)
    Qbar = Qbar + Ah @ Bbar.T                         # B = Q^T Ah
    Ahbar = Q @ Bbar
    for i in range(q, 0, -1):
        Ybar = _qr_vjp(Qs[i], Rs[i], Qbar)            # Q_i R_i = Y_i
        Ahbar += Ybar @ Zs[i - 1].T                   # Y_i = Ah Z_i
        Zbar = Ah.T @ Ybar
        Ahbar += Qs[i - 1] @ Zbar.T                   # Z_i = Ah^T Q_{i-1}
        Qbar = Ah @ Zbar
    Ybar = _qr_vjp(Qs[0], Rs[0], Qbar)                # Q_0 R_0 = Y_0
    Ahbar += Ybar @ Omega.T                           # Y_0 = Ah Omega
    Abar = Ahbar.T if transposed else Ahbar
    X = Xh.T if transposed else Xh
    return np.ascontiguousarray(Abar), float(taubar), np.ascontiguousarray(X)


def frsvt_directional_fd(A: np.ndarray, tau: float, l: int, q: int, seed: int, stream: int,
                         Xbar: np.ndarray, E: np.ndarray, h: float = 1e-3, dtau: float = 0.0) -> float:
    """Central difference of <Xbar, FRSVT(A, tau)> along (E, dtau) with the same Omega.

    The FRSVT map with a fixed Omega is what a backward pass of Alg. 1 differentiates; it is
    smooth where no singular value of B sits at tau (the shrinkage kink) and the sketch keeps
    its rank.
    """
    fp = frsvt(A + h * E, tau + h * dtau, l, q, seed, stream).X
    fm = frsvt(A - h * E, tau - h * dtau, l, q, seed, stream).X
    return float(np.sum(Xbar * (fp - fm)) / (2.0 * h))
