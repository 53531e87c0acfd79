"""Robust PCA by the inexact augmented Lagrange multiplier method, FP64 (test infrastructure only).

The paper's host algorithm for its RPCA experiments (Sec. 4.1, "Robust PCA
test") is the inexact ALM of its reference [18], whose steps the paper does not
print.  This oracle follows one reading of it, stated here in full:

    min ||L||_* + lam ||S||_1   s.t.  O = L + S,   lam = 1 / sqrt(max(m, n))
    init:  S = 0,  Y = O / max(||O||_2, ||O||_inf / lam),  mu = mu0 = 1.25 / ||O||_2,
           mu_bar = 1e7 * mu0
    each iteration k:
        L  = SVT_{1/mu}(O - S + Y / mu)          (exact SVT or FRSVT)
        S  = shrink_{lam/mu}(O - L + Y / mu)
        Z  = O - L - S
        Y  = Y + mu Z
        mu = min(rho mu, mu_bar)
        stop when ||Z||_F / ||O||_F < tol (unless a fixed iteration count is asked for)

||O||_inf is the largest absolute entry.  The FRSVT variant draws Omega from
stream k at iteration k and propagates the basis across iterations (Alg. 1
range propagation).

Parity status: partly pinned.  The fixed point is the unique RPCA optimum
(a convex problem), so exact-SVT and FRSVT runs must agree with each other and
recover planted low-rank + sparse data; the paper's Table 5 reports equal
iteration counts for exact SVD and FRSVT-RP, which the tests mirror.  The exact
constants of [18] are not in the paper and remain a reading.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import svt as svt_mod


@dataclass
class RPCAResult:
    L: np.ndarray
    S: np.ndarray
    Y: np.ndarray
    mu: float
    iters: int
    history: list = field(default_factory=list)     # ||Z||_F / ||O||_F per iteration
    ranks: list = field(default_factory=list)       # #{sigma > 1/mu} per iteration
    ls: list = field(default_factory=list)          # sampling rates l_i (adaptive rank prediction)


def spectral_norm(O: np.ndarray) -> float:
    """||O||_2 (largest singular value) from the oracle's Jacobi SVD."""
    from .linalg import jacobi_svd
    return float(jacobi_svd(O)[1][0]) if O.size else 0.0


def ialm_init(O: np.ndarray, lam: float, normO2: float | None = None):
    """Initial dual variable and penalty: (Y0, mu0)."""
    if normO2 is None:
        normO2 = spectral_norm(O)
    norm_inf = float(np.max(np.abs(O))) / lam
    Y0 = O / max(normO2, norm_inf)
    mu0 = 1.25 / normO2
    return Y0, mu0


def predict_rank(r: int, l: int, n: int, a: int, rho_ap: float, b: int) -> int:
    """Adaptive rank prediction, Eq. 7 (Sec. 2.3): the next sampling rate from the current rank
    estimate r = #{sigma_i > tau} and sampling rate l, for the short side n.  Over-sample by a
    when r < l, by ceil(rho_ap n) otherwise (the rank may still be growing); at most b."""
    p = a if r < l else int(np.ceil(rho_ap * n))
    return int(min(r + p, b))


def ialm_rpca(O: np.ndarray, lam: float | None = None, mu0: float | None = None,
              rho: float = 1.5, mu_bar: float | None = None, tol: float = 1e-7,
              max_iter: int = 500, method: str = "exact", l: int = 0, q: int = 0,
              seed: int = 0, range_prop: bool = True, fixed_iters: int | None = None,
              normO2: float | None = None, rank_tol: float = 1e-12,
              ap: dict | None = None, partial_k: int = 0, orth_last: bool = False) -> RPCAResult:
    """Inexact ALM RPCA.  With ``ap`` (keys a, rho, gamma; FRSVT with range propagation) the
    sampling rate follows the adaptive rank prediction of Eq. 7: l_0 = ceil(0.1 b), b =
    ceil(gamma n) for the short side n, l_{i+1} = predict_rank(r_i, l_i, ...); the propagated
    basis keeps min(r_i, l_{i+1} - a) columns (r_i in the paper, capped so that at least a new
    Gaussian columns are drawn) and the call draws l_{i+1} - keep new ones.  The sampling rates
    used are recorded in ``res.ls``.  ``orth_last`` is passed to every FRSVT call (orthonormalise
    only after the last power step, Sec. 2.5)."""
    O = np.asarray(O, dtype=np.float64)
    m, n = O.shape
    if lam is None:
        lam = 1.0 / np.sqrt(max(m, n))
    Y, mu_init = ialm_init(O, lam, normO2)
    mu = mu_init if mu0 is None else mu0
    if mu_bar is None:
        mu_bar = 1e7 * mu
    S = np.zeros_like(O)
    L = np.zeros_like(O)
    normO = np.linalg.norm(O)
    Qt = None
    res = RPCAResult(L, S, Y, mu, 0)
    n_iter = fixed_iters if fixed_iters is not None else max_iter
    ns = min(m, n)
    if ap is not None:
        b = int(np.ceil(ap["gamma"] * ns))
        l_cur = max(1, int(np.ceil(0.1 * b)))
        res.ls = []
    for k in range(n_iter):
        Ain = O - S + Y / mu
        if method == "exact":
            if partial_k > 0:
                L = svt_mod.psvt(Ain, 1.0 / mu, partial_k)
                r = int(np.linalg.matrix_rank(L))
            else:
                L, r = svt_mod.exact_svt(Ain, 1.0 / mu)
        elif method == "frsvt":
            l_k = l if ap is None else l_cur
            out = svt_mod.frsvt(Ain, 1.0 / mu, l_k, q, seed, k,
                                Q_prev=Qt if range_prop else None, rank_tol=rank_tol, partial_k=partial_k,
                                orth_last=orth_last)
            L, r = out.X, out.r
            if ap is None:
                Qt = out.Q_tilde
            else:
                res.ls.append(l_k)
                l_cur = predict_rank(r, l_k, ns, ap["a"], ap["rho"], b)
                keep = max(0, min(r, l_cur - ap["a"]))
                Qt = np.ascontiguousarray(out.extra["QV"][:, :keep])
        else:
            raise ValueError(method)
        S = svt_mod.soft(O - L + Y / mu, lam / mu)
        Z = O - L - S
        Y = Y + mu * Z
        mu = min(rho * mu, mu_bar)
        err = float(np.linalg.norm(Z) / normO) if normO > 0 else 0.0
        res.history.append(err)
        res.ranks.append(r)
        res.iters = k + 1
        if fixed_iters is None and err < tol:
            break
    res.L, res.S, res.Y, res.mu = L, S, Y, mu
    return res
