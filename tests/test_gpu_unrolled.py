"""Unrolled RPCA with learnable tau_k, mu_k: GPU gradients against FP64 central differences.

The FP64 reference runs the same unrolled iALM with the oracle's FRSVT (same Omega streams) and
differentiates the loss by central differences in each parameter.  Every step's tau_k and mu_k is
compared at 1e-3; each test asserts how many parameters it compared and that no step's
threshold sits near a singular value of B (the shrinkage kink, where the map is not
differentiable).

The evaluation points keep the iteration away from convergence (penalty growth rho = 1.2): at a
converged step the cotangent 2 (L_K - L_true) is the tiny recovery error, whose FP32 rounding
(about 1e-6 of L) is then a visible fraction of it, and no FP32 pipeline can match an FP64
gradient to 1e-3 there.  With a full basis (l = n) FRSVT is the exact SVT, and the GPU gradient is
checked against central differences of the exact-SVT pipeline.
"""
import numpy as np
import pytest

from oracle import svt
from paper_1509_00296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 13
RTOL = 1e-3


def _oracle_loss(O, Lt, ys, tau, mu, lam, l, q, exact=False, gaps=None):
    """sum_b ||L_K(b) - L_true(b)||^2 of the unrolled iALM in FP64 (Y_0 = ys_b O_b)."""
    total = 0.0
    for b in range(O.shape[0]):
        S = np.zeros_like(O[b])
        Y = ys[b] * O[b]
        L = None
        for k in range(len(tau)):
            A = O[b] - S + Y / mu[k]
            if exact:
                L = svt.exact_svt(A, tau[k])[0]
            else:
                res = svt.frsvt(A, tau[k], l, q, SEED, k)
                L = res.X
                if gaps is not None:             # distance of the nearest sigma of B to tau_k
                    gaps.append(float(np.min(np.abs(res.sigma - tau[k])) / tau[k]))
            T = O[b] - L + Y / mu[k]
            S = svt.soft(T, lam / mu[k])
            Y = Y + mu[k] * (O[b] - L - S)
        total += float(np.sum((L - Lt[b]) ** 2))
    return total


def _y0_scales(O, lam):
    return [1.0 / max(np.linalg.norm(o, 2), np.abs(o).max() / lam) for o in O]


def _run(m, n, steps, l, q, batch, batch_seed, rho, exact_ref=False, tau_scale=1.0):
    """GPU loss and gradients against the FP64 oracle; returns the number of parameters compared."""
    from paper_1509_00296_gb300.unrolled import RPCAUnrolled
    O3, L3, _ = synth.unrolled_batch(seed=batch_seed, batch=batch, m=m, n=n)
    O = O3.astype(np.float32).astype(np.float64)
    Lt = L3.astype(np.float32).astype(np.float64)
    lam = 1.0 / np.sqrt(m)
    ys = _y0_scales(O, lam)
    mu0 = 1.25 / np.linalg.norm(O[0], 2)
    net = RPCAUnrolled(m, n, steps=steps, l=l, q=q, lam=lam, mu0=mu0, rho=rho, seed=SEED)
    with torch.no_grad():
        net.tau.mul_(tau_scale)
    Od = torch.from_numpy(O.astype(np.float32)).cuda()
    loss = net.loss(Od, torch.from_numpy(Lt.astype(np.float32)).cuda(), y0_scale=ys)
    loss.backward()
    gt = net.tau.grad.cpu().numpy().astype(np.float64)
    gm = net.mu.grad.cpu().numpy().astype(np.float64)
    tau = net.tau.detach().cpu().numpy().astype(np.float64)
    mu = net.mu.detach().cpu().numpy().astype(np.float64)
    args = (O, Lt, ys)
    gaps = []
    ref = _oracle_loss(*args, tau, mu, lam, l, q, exact=exact_ref, gaps=None if exact_ref else gaps)
    if gaps:
        print("relative distance of the nearest singular value of B to tau_k:", np.round(gaps, 4))
        assert min(gaps) > 1e-3, gaps                      # no step sits on the shrinkage kink
    assert abs(float(loss.detach()) - ref) <= RTOL * max(ref, 1e-6), (float(loss.detach()), ref)
    compared = 0
    for name in ("tau", "mu"):
        base = tau if name == "tau" else mu
        got = gt if name == "tau" else gm
        fds = []
        for k in range(steps):
            h = 1e-5 * base[k]
            p, mq = base.copy(), base.copy()
            p[k] += h
            mq[k] -= h
            if name == "tau":
                fds.append((_oracle_loss(*args, p, mu, lam, l, q, exact_ref) -
                            _oracle_loss(*args, mq, mu, lam, l, q, exact_ref)) / (2 * h))
            else:
                fds.append((_oracle_loss(*args, tau, p, lam, l, q, exact_ref) -
                            _oracle_loss(*args, tau, mq, lam, l, q, exact_ref)) / (2 * h))
        floor = 1e-7 * max(abs(f) for f in fds)      # a threshold above every singular value: both exactly 0
        for k, fd in enumerate(fds):
            print(f"{name}_{k}: gpu {got[k]:.6g} fd {fd:.6g} rel {abs(got[k] - fd) / max(abs(fd), 1e-300):.2e}")
            assert abs(got[k] - fd) <= RTOL * abs(fd) + floor, (name, k, got[k], fd)
            compared += 1
    return compared


def test_unrolled_small_all_parameters():
    assert _run(256, 96, 4, 8, 1, batch=1, batch_seed=91, rho=1.2) == 8


def test_unrolled_batch_of_two_all_parameters():
    """Two problems in one library call: the gradients are those of the summed loss."""
    assert _run(256, 96, 3, 8, 1, batch=2, batch_seed=95, rho=1.2) == 6


def test_unrolled_full_size_all_parameters():
    """One 2048 x 512 matrix of the unrolled batch, 10 steps, l = 16, q = 1: all 20 parameters.
    The thresholds are evaluated at 3 / mu_k: at 1 / mu_k every step keeps all eight signal singular
    values, d loss / d tau_k is a near-cancelling projection of 1e-5 .. 1e-3 of the other terms,
    and FP32 rounding of the backward alone is about 1e-3 of it."""
    assert _run(2048, 512, 10, 16, 1, batch=1, batch_seed=1005, rho=1.2, tau_scale=3.0) == 20


def test_unrolled_full_basis_equals_exact_svd_gradient():
    """l = n: FRSVT is the exact SVT, so the gradient matches central differences of the
    exact-SVT pipeline (the FP64 oracle's exact-SVD reference gradient) at 1e-3."""
    assert _run(128, 32, 3, 32, 1, batch=1, batch_seed=97, rho=1.2, exact_ref=True) == 6


def test_unrolled_concurrent_batch_matches_serial():
    """The batch run on child handles with their own streams (problem_streams) gives the loss and
    gradients of the one-stream run: the same kernels per problem, only the order of the
    per-problem gradient sums differs."""
    import torch
    from paper_1509_00296_gb300.unrolled import RPCAUnrolled
    O3, L3, _ = synth.unrolled_batch(seed=77, batch=3, m=512, n=128)
    Od = torch.from_numpy(O3.astype(np.float32)).cuda()
    Lt = torch.from_numpy(L3.astype(np.float32)).cuda()
    out = []
    for streams in (0, 2):
        net = RPCAUnrolled(512, 128, steps=4, l=8, q=1, mu0=0.01, rho=1.2, seed=SEED, streams=streams)
        loss = net.loss(Od, Lt)
        loss.backward()
        out.append((float(loss.detach()), net.tau.grad.cpu().numpy(), net.mu.grad.cpu().numpy()))
    (l0, t0, m0), (l1, t1, m1) = out
    assert abs(l0 - l1) <= 1e-6 * abs(l0)
    assert np.allclose(t0, t1, rtol=1e-5, atol=1e-7 * np.abs(t0).max())
    assert np.allclose(m0, m1, rtol=1e-5, atol=1e-7 * np.abs(m0).max())
