"""Low-rank representation (Table 6, Type A) by the inexact augmented Lagrange multiplier
method, FP64 (test infrastructure only).

Problem (Table 6, Type A):

    min ||L||_* + lam ||S||_{2,1}   s.t.   O = Z L + S,

with ||S||_{2,1} the sum of the column 2-norms and the dictionary Z (the data itself, Z = O,
unless another is given).  The paper states the objective and that iALM solves it; the
splitting below is one reading of that solver, written out here in full: an auxiliary
J = L carries the nuclear norm, so each iteration applies SVT once, to an n x n matrix
(the step FRSVT replaces), plus a linear solve and a column shrinkage:

    init:  L = J = 0, S = 0, Y1 = 0 (d x n), Y2 = 0 (n x n), mu = mu0
    each iteration k:
        J  = SVT_{1/mu}(L + Y2 / mu)                                   (exact SVT or FRSVT)
        L  = (I + Z^T Z)^{-1} (Z^T (O - S) + J + (Z^T Y1 - Y2) / mu)
        S  = colshrink_{lam/mu}(O - Z L + Y1 / mu)
        Y1 = Y1 + mu (O - Z L - S),   Y2 = Y2 + mu (L - J)
        mu = min(rho mu, mu_max)
        stop when max(||O - Z L - S||_inf, ||L - J||_inf) < tol (unless a fixed count is asked)

colshrink_t(Q) scales column q_i by max(0, 1 - t / ||q_i||) (the proximal map of t ||.||_{2,1}).
Defaults (a reading; the paper gives none): mu0 = 1e-6, rho = 1.1, mu_max = 1e10, tol = 1e-8.  The
penalty grows geometrically, and the iterate settles at a feasible point whose objective exceeds
the optimum by an amount that shrinks with rho - 1 (about 6e-5 relative at rho = 1.1, 2e-3 at
rho = 1.2 on the pinned problem); the optimality pin runs at rho = 1.02.

Pinned by: the proximal map against its optimality conditions and random perturbations; the closed
form of the noiseless problem (min ||L||_* s.t. O = O L has the solution V V^T for the skinny
SVD O = U S V^T, the shape-interaction matrix); the block-diagonal structure of L for
independent subspaces; feasibility and the S-step optimality of the returned point (Y1 in lam
times the l2,1 subdifferential at S); the optimal value reached by an independent two-block
linearised ADMM; the corrupted columns carrying the largest columns of S; and FRSVT with a full
basis reproducing the exact-SVT iteration (with range propagation and l = 12 the same fixed point).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import svt as svt_mod


def colshrink(Q: np.ndarray, t: float) -> np.ndarray:
    """Proximal map of t ||.||_{2,1}: column i becomes max(0, 1 - t / ||q_i||) q_i."""
    Q = np.asarray(Q, dtype=np.float64)
    nrm = np.linalg.norm(Q, axis=0)
    scale = np.where(nrm > t, 1.0 - t / np.where(nrm > 0.0, nrm, 1.0), 0.0)
    return Q * scale


def l21(S: np.ndarray) -> float:
    return float(np.linalg.norm(np.asarray(S, dtype=np.float64), axis=0).sum())


@dataclass
class LRRResult:
    L: np.ndarray
    S: np.ndarray
    J: np.ndarray
    Y1: np.ndarray
    Y2: np.ndarray
    mu: float
    iters: int
    history: list = field(default_factory=list)


def lrr_ialm(O: np.ndarray, lam: float, Z: np.ndarray | None = None, method: str = "exact", l: int = 0,
             q: int = 1, seed: int = 0, range_prop: bool = True, mu0: float = 1e-6, rho: float = 1.1,
             mu_max: float = 1e10, tol: float = 1e-8, max_iter: int = 1000,
             fixed_iters: int | None = None) -> LRRResult:
    """Inexact ALM for min ||L||_* + lam ||S||_{2,1} s.t. O = Z L + S (see the module text).
    With method="frsvt" the J step is Alg. 1 with l columns and q power steps, Omega from stream k
    at iteration k and the basis propagated across iterations when range_prop."""
    O = np.asarray(O, dtype=np.float64)
    Z = O if Z is None else np.asarray(Z, dtype=np.float64)
    d, n = O.shape
    p = Z.shape[1]
    ZtZ = Z.T @ Z
    inv = np.linalg.inv(np.eye(p) + ZtZ)
    L = np.zeros((p, n))
    J = np.zeros((p, n))
    S = np.zeros((d, n))
    Y1 = np.zeros((d, n))
    Y2 = np.zeros((p, n))
    mu = mu0
    Qt = None
    res = LRRResult(L, S, J, Y1, Y2, mu, 0)
    n_iter = fixed_iters if fixed_iters is not None else max_iter
    for k in range(n_iter):
        M = L + Y2 / mu
        if method == "exact":
            J, _ = svt_mod.exact_svt(M, 1.0 / mu)
        elif method == "frsvt":
            out = svt_mod.frsvt(M, 1.0 / mu, l, q, seed, k, Q_prev=Qt if range_prop else None)
            J = out.X
            Qt = out.Q_tilde
        else:
            raise ValueError(method)
        L = inv @ (Z.T @ (O - S) + J + (Z.T @ Y1 - Y2) / mu)
        ZL = Z @ L
        S = colshrink(O - ZL + Y1 / mu, lam / mu)
        R1 = O - ZL - S
        R2 = L - J
        Y1 = Y1 + mu * R1
        Y2 = Y2 + mu * R2
        mu = min(rho * mu, mu_max)
        err = max(float(np.abs(R1).max(initial=0.0)), float(np.abs(R2).max(initial=0.0)))
        res.history.append(err)
        res.iters = k + 1
        if fixed_iters is None and err < tol:
            break
    res.L, res.S, res.J, res.Y1, res.Y2, res.mu = L, S, J, Y1, Y2, mu
    return res
