"""Unrolled RPCA with learnable tau_k, mu_k: GPU gradients against FP64 central differences.

The FP64 reference runs the same unrolled iALM with the oracle's FRSVT (same Omega streams)
and differentiates the loss by central differences in each parameter.  The same pipeline with
the exact SVT gives the exact-SVD reference gradient, reported as an approximation gap.
"""
import numpy as np
import pytest

from oracle import svt
from paper_1509_00296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 13


def _oracle_loss(O, Lt, Y0, tau, mu, lam, l, q, exact=False, gaps=None):
    S = np.zeros_like(O)
    Y = Y0.copy()
    L = None
    for k in range(len(tau)):
        A = O - S + Y / mu[k]
        if exact:
            L = svt.exact_svt(A, tau[k])[0]
        else:
            res = svt.frsvt(A, tau[k], l, q, SEED, k)
            L = res.X
            if gaps is not None:                 # distance of the nearest sigma of B to tau_k
                gaps.append(float(np.min(np.abs(res.sigma - tau[k])) / tau[k]))
        T = O - L + Y / mu[k]
        S = svt.soft(T, lam / mu[k])
        Y = Y + mu[k] * (O - L - S)
    return float(np.sum((L - Lt) ** 2))


def _run(m, n, steps, l, q, batch_seed, n_fd, exact_gap, picks=None):
    from paper_1509_00296_gb300.unrolled import RPCAUnrolled
    O3, L3, _ = synth.unrolled_batch(seed=batch_seed, batch=1, m=m, n=n)
    O, Lt = O3[0].astype(np.float32), L3[0].astype(np.float32)
    lam = 1.0 / np.sqrt(m)
    norm2 = np.linalg.norm(O.astype(np.float64), 2)
    Y0 = (O.astype(np.float64) / max(norm2, np.abs(O).max() / lam)).astype(np.float32)
    mu0 = 1.25 / norm2
    net = RPCAUnrolled(m, n, steps=steps, l=l, q=q, lam=lam, mu0=mu0, rho=1.5, seed=SEED)
    Od = torch.from_numpy(O).cuda()
    L = net.forward_one(Od, Y0=torch.from_numpy(Y0).cuda())
    loss = torch.sum((L - torch.from_numpy(Lt).cuda()) ** 2)
    loss.backward()
    gt, gm = net.tau.grad.cpu().numpy().astype(np.float64), net.mu.grad.cpu().numpy().astype(np.float64)
    tau = net.tau.detach().cpu().numpy().astype(np.float64)
    mu = net.mu.detach().cpu().numpy().astype(np.float64)
    args = (O.astype(np.float64), Lt.astype(np.float64), Y0.astype(np.float64))
    gaps = []
    ref = _oracle_loss(*args, tau, mu, lam, l, q, gaps=gaps)
    print("relative distance of the nearest singular value of B to tau_k, per step:", np.round(gaps, 5))
    assert abs(float(loss) - ref) <= 1e-3 * max(ref, 1e-6), (float(loss), ref)
    # the map is not differentiable where a singular value of B sits at tau_k (the shrinkage kink):
    # parameters of the steps from the first near-kink step on are not compared
    first_kink = next((k for k, g in enumerate(gaps) if g < 1e-3), steps)
    if picks is None:
        picks = [("tau", k, 1e-3) for k in range(first_kink)] + [("mu", k, 1e-3) for k in range(first_kink)]
        if n_fd < len(picks):
            picks = [picks[i] for i in np.linspace(0, len(picks) - 1, n_fd).astype(int)]
    picks = [p for p in picks if p[1] < first_kink]
    for name, k, rtol in picks:
        base = tau if name == "tau" else mu
        h = 1e-5 * base[k]
        p, mq = base.copy(), base.copy()
        p[k] += h
        mq[k] -= h
        if name == "tau":
            fd = (_oracle_loss(*args, p, mu, lam, l, q) - _oracle_loss(*args, mq, mu, lam, l, q)) / (2 * h)
            got = gt[k]
        else:
            fd = (_oracle_loss(*args, tau, p, lam, l, q) - _oracle_loss(*args, tau, mq, lam, l, q)) / (2 * h)
            got = gm[k]
        print(f"{name}_{k}: gpu {got:.6g} fd {fd:.6g} rel {abs(got - fd) / abs(fd):.2e}")
        assert abs(got - fd) <= rtol * abs(fd), (name, k, got, fd)
    if exact_gap:
        ge = []
        for k in range(steps):
            h = 1e-5 * tau[k]
            p, mq = tau.copy(), tau.copy()
            p[k] += h
            mq[k] -= h
            ge.append((_oracle_loss(*args, p, mu, lam, l, q, True) - _oracle_loss(*args, mq, mu, lam, l, q, True))
                      / (2 * h))
        gap = np.linalg.norm(gt - np.array(ge)) / max(np.linalg.norm(ge), 1e-30)
        print(f"d loss / d tau: relative gap of the FRSVT pipeline to the exact-SVD pipeline {gap:.3e}")
        assert np.isfinite(gap)


def test_unrolled_small_all_parameters():
    _run(256, 96, 4, 8, 1, batch_seed=91, n_fd=8, exact_gap=True)


def test_unrolled_full_size_sampled_parameters():
    """One 2048 x 512 matrix of the unrolled batch, 10 steps, l = 16, q = 1.

    Steps before convergence are compared at 1e-3.  Near convergence (the last steps) the true
    gradients shrink towards the size of the perturbation that the FP32 forward's rounding causes
    in the final error L - L_true (d loss / d tau_K = -2 sum_i u_i^T (L - L_true) v_i), so the
    last step is only bounded (5e-2); the adjoint of the FRSVT map itself is pinned at this size
    at 1e-3 (test_gpu_adjoint)."""
    picks = [("mu", 0, 1e-3), ("mu", 2, 1e-3), ("mu", 4, 1e-3), ("tau", 0, 1e-3), ("mu", 9, 5e-2)]
    _run(2048, 512, 10, 16, 1, batch_seed=1005, n_fd=len(picks), exact_gap=False, picks=picks)
