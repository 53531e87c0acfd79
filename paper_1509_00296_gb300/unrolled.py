"""Unrolled inexact-ALM RPCA with learnable per-step thresholds (the differentiable workload).

K iALM steps (the iteration of the cited inexact ALM, Sec. 4.1) are unrolled into a network
whose step k has its own SVT threshold tau_k and penalty mu_k, both learnable:

    A_k = O - S + Y / mu_k
    L   = FRSVT_{tau_k}(A_k)                      (Alg. 1, fixed Omega stream k)
    S   = shrink_{lambda / mu_k}(O - L + Y / mu_k)
    Y   = Y + mu_k (O - L - S)

starting from S = 0 and Y = O / max(||O||_2, ||O||_inf / lambda).  The whole batch and every step
run in the library (rpca_unrolled_forward / rpca_unrolled_backward: the FRSVT, its adjoint and
fused kernels for the shrinkage, the multiplier update and their adjoints); this module only
keeps the parameters and wires the two calls into a torch.autograd.Function.  The default
schedule is the iALM one: mu_k = mu_0 rho^k, tau_k = 1 / mu_k.
"""
from __future__ import annotations

import math

from . import frsvt as fr


def _torch():
    import torch
    return torch


def _function():
    torch = _torch()

    class UnrolledRPCA(torch.autograd.Function):
        """L_K of the unrolled iALM for a batch; gradients with respect to tau and mu."""

        @staticmethod
        def forward(ctx, tau, mu, Ob, handle, lam, l, y0_scale):
            t = [float(v) for v in tau.detach().cpu()]
            mv = [float(v) for v in mu.detach().cpu()]
            L, saved = handle.unrolled_forward(Ob, y0_scale, t, mv, lam, l)
            ctx.save_for_backward(Ob, saved)
            ctx.meta = (handle, lam, l, y0_scale, t, mv)
            return L

        @staticmethod
        def backward(ctx, dL):
            Ob, saved = ctx.saved_tensors
            handle, lam, l, y0_scale, t, mv = ctx.meta
            dtau, dmu = handle.unrolled_backward(Ob, y0_scale, t, mv, lam, l, saved, dL)
            return dtau, dmu, None, None, None, None, None

    return UnrolledRPCA


class RPCAUnrolled:
    """Learnable unrolled RPCA over a batch of m x n matrices (m >= n, n % 4 == 0).

    Parameters (torch tensors with requires_grad): ``tau`` and ``mu`` of shape (K,).
    """

    def __init__(self, m: int, n: int, steps: int = 10, l: int = 16, q: int = 1, lam: float | None = None,
                 mu0: float = 1.0, rho: float = 1.5, seed: int = 0, device="cuda", streams: int = 8):
        """streams: concurrent problems of a batch (child handles of the library, each with its own
        CUDA stream and workspace); 0 or 1 runs them one after another."""
        torch = _torch()
        self.m, self.n, self.K, self.l = m, n, steps, l
        self.lam = lam if lam is not None else 1.0 / math.sqrt(max(m, n))
        self.handle = fr.Handle(m, n, l, q=q, seed=seed, adjoint=True, range_prop=False,
                                problem_streams=streams if streams > 1 else 0)
        mu = torch.tensor([mu0 * rho ** k for k in range(steps)], dtype=torch.float32, device=device)
        self.mu = mu.clone().requires_grad_(True)
        self.tau = (1.0 / mu).clone().requires_grad_(True)

    def parameters(self):
        return [self.tau, self.mu]

    def dual_scales(self, Ob):
        """y0 scales 1 / max(||O_b||_2, ||O_b||_inf / lambda) of a batch (computed by the library:
        a spectral-norm estimate per matrix, a few milliseconds each)."""
        return self.handle.unrolled_init(Ob.contiguous(), self.lam)

    def forward(self, Ob, y0_scale=None):
        """Ob: (B, m, n) float32 CUDA.  Returns L_K as a (B, m, n) tensor.  Without y0_scale the
        scales are those of Ob, computed on the first call for a given tensor and reused while
        the same, unmodified tensor comes back (they depend on the data only)."""
        Ob = Ob.contiguous()
        if y0_scale is None:
            key = (Ob.data_ptr(), tuple(Ob.shape), Ob._version)
            if getattr(self, "_scales_key", None) != key:
                self._scales = self.dual_scales(Ob)
                self._scales_key = key
            ys = list(self._scales)
        else:
            ys = list(y0_scale)
        return _function().apply(self.tau, self.mu, Ob, self.handle, self.lam, self.l, ys)

    def loss(self, Ob, Lb_true, y0_scale=None):
        """The training objective of the workload, sum_b ||L_K(b) - L_true(b)||_F^2."""
        torch = _torch()
        return torch.sum((self.forward(Ob, y0_scale) - Lb_true) ** 2)
