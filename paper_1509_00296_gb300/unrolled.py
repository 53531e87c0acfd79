"""Unrolled inexact-ALM RPCA with learnable per-step thresholds (the differentiable workload).

K iALM steps (the iteration of the cited inexact ALM, Sec. 4.1) are unrolled into a network
whose step k has its own SVT threshold tau_k and penalty mu_k, both learnable:

    A_k = O - S + Y / mu_k
    L   = FRSVT_{tau_k}(A_k)                      (Alg. 1, fixed Omega stream k)
    S   = shrink_{lambda / mu_k}(O - L + Y / mu_k)
    Y   = Y + mu_k (O - L - S)

starting from S = 0 and Y = O / max(||O||_2, ||O||_inf / lambda).  The SVT and its gradient
(with respect to A_k and tau_k) run in the library (frsvt_svt_save / frsvt_backward); the
elementwise shrinkage and dual update are torch operations on the GPU, differentiated by
autograd.  The default schedule is the iALM one: mu_k = mu_0 rho^k, tau_k = 1 / mu_k.
"""
from __future__ import annotations

import math

from . import frsvt as fr


def _torch():
    import torch
    return torch


class RPCAUnrolled:
    """Learnable unrolled RPCA over a batch of m x n matrices (m >= n).

    Parameters (torch tensors with requires_grad): ``tau`` and ``mu`` of shape (K,).
    """

    def __init__(self, m: int, n: int, steps: int = 10, l: int = 16, q: int = 1, lam: float | None = None,
                 mu0: float = 1.0, rho: float = 1.5, seed: int = 0, device="cuda"):
        torch = _torch()
        self.m, self.n, self.K, self.l = m, n, steps, l
        self.lam = lam if lam is not None else 1.0 / math.sqrt(max(m, n))
        self.handle = fr.Handle(m, n, l, q=q, seed=seed, adjoint=True, range_prop=False)
        mu = torch.tensor([mu0 * rho ** k for k in range(steps)], dtype=torch.float32, device=device)
        self.mu = mu.clone().requires_grad_(True)
        self.tau = (1.0 / mu).clone().requires_grad_(True)

    def parameters(self):
        return [self.tau, self.mu]

    def dual_init(self, O):
        """Y_0 = O / max(||O||_2, ||O||_inf / lambda) with ||O||_2 from the library's power method."""
        norm2 = self.handle.spectral_norm(O)
        return O / max(norm2, float(O.abs().max()) / self.lam)

    def forward_one(self, O, Y0=None):
        torch = _torch()
        Y = self.dual_init(O) if Y0 is None else Y0
        S = torch.zeros_like(O)
        L = None
        for k in range(self.K):
            mu, tau = self.mu[k], self.tau[k]
            A = O - S + Y / mu
            L = fr.frsvt_svt_autograd(A, tau, self.handle, self.l, k)
            T = O - L + Y / mu
            S = torch.sign(T) * torch.relu(T.abs() - self.lam / mu)
            Y = Y + mu * (O - L - S)
        return L

    def forward(self, Ob):
        """Ob: (B, m, n) float32 CUDA.  Returns the list of L_K per batch element."""
        return [self.forward_one(Ob[b]) for b in range(Ob.shape[0])]

    def loss(self, Ob, Lb_true):
        torch = _torch()
        Ls = self.forward(Ob)
        return sum(torch.sum((L - Lt) ** 2) for L, Lt in zip(Ls, Lb_true))
