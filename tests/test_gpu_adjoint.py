"""Adjoint of the FRSVT map (frsvt_svt_save / frsvt_backward) against the FP64 oracle.

The FRSVT map with a fixed Omega is differentiated; dA and dtau are compared entry by entry
with the oracle's FP64 adjoint of the same map (``oracle.svt.frsvt_vjp``, pinned by entrywise
central differences), with tau halfway across a wide gap of B's singular values.  The
exact-SVD gradient is reported beside it.
"""
import numpy as np
import pytest

from oracle import svt
from paper_1509_00296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 21


def _fr():
    from paper_1509_00296_gb300 import frsvt as fr
    return fr


def _case(m, n, rank, seed, noise=0.05):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n)) / np.sqrt(rank)
    A += noise * rng.standard_normal((m, n))
    return A.astype(np.float32)


def _tau_between(A, l, q, stream):
    """tau halfway between two well separated singular values of the oracle's B."""
    d = svt.frsvt(A.astype(np.float64), 0.0, l, q, SEED, stream).sigma
    gaps = d[:-1] - d[1:]
    i = int(np.argmax(gaps[: max(1, len(gaps) // 2)]))
    return float(0.5 * (d[i] + d[i + 1]))


def _check_entrywise(dA, dtau, ref_A, ref_tau):
    """dA entry by entry against the oracle's FRSVT-map adjoint: 1e-3 in relative Frobenius norm and in
    the largest entry error relative to the largest entry."""
    err_f = np.linalg.norm(dA - ref_A) / np.linalg.norm(ref_A)
    err_max = np.max(np.abs(dA - ref_A)) / np.max(np.abs(ref_A))
    assert err_f <= 1e-3, err_f
    assert err_max <= 1e-3, err_max
    assert abs(dtau - ref_tau) <= 1e-3 * max(abs(ref_tau), 1.0), (dtau, ref_tau)
    return err_f, err_max


@pytest.mark.parametrize("shape,l,q", [((300, 120), 8, 1), ((257, 96), 12, 2), ((300, 120), 16, 0)])
def test_adjoint_matches_oracle_vjp_entrywise(shape, l, q):
    """frsvt_backward's dA and dtau against the FP64 oracle frsvt_vjp with the same Omega, every entry."""
    fr = _fr()
    m, n = shape
    A = _case(m, n, 5, seed=31 + m)
    stream = 3
    tau = _tau_between(A, l, q, stream)
    h = fr.Handle(m, n, 16, q=q, seed=SEED, adjoint=True)
    Ad = torch.from_numpy(A).cuda()
    X, saved = h.svt_save(Ad, tau, l, stream)
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    Xbar = rng.standard_normal((m, n)).astype(np.float32)
    ref_A, ref_tau, ref_X = svt.frsvt_vjp(A.astype(np.float64), tau, l, q, SEED, stream, Xbar.astype(np.float64))
    assert np.linalg.norm(X.cpu().numpy() - ref_X) <= 1e-4 * np.linalg.norm(ref_X)
    dA, dtau = h.backward(saved, Ad, tau, l, stream, torch.from_numpy(Xbar).cuda())
    torch.cuda.synchronize()
    assert h.info().device_status == 0
    dA = dA.cpu().numpy().astype(np.float64)
    err_f, err_max = _check_entrywise(dA, float(dtau.item()), ref_A, ref_tau)
    if shape == (300, 120) and q == 1:
        Ae, te = svt.svt_vjp(A.astype(np.float64), tau, Xbar.astype(np.float64))
        gap = np.linalg.norm(dA - Ae) / np.linalg.norm(Ae)
        print(f"entrywise error {err_f:.2e} (max {err_max:.2e}); relative gap to the exact-SVD gradient "
              f"{gap:.3e} (dtau {float(dtau.item()):.4g} vs {te:.4g})")


def test_adjoint_matches_oracle_fd_direction():
    """The oracle's adjoint itself agrees with a central difference of its FRSVT map on the GPU case."""
    m, n, l, q = 300, 120, 8, 1
    A = _case(m, n, 5, seed=31 + m).astype(np.float64)
    tau = _tau_between(A.astype(np.float32), l, q, 3)
    rng = np.random.default_rng(77)
    Xbar = rng.standard_normal((m, n))
    ref_A, _, _ = svt.frsvt_vjp(A, tau, l, q, SEED, 3, Xbar)
    E = rng.standard_normal((m, n))
    fd = svt.frsvt_directional_fd(A, tau, l, q, SEED, 3, Xbar, E)
    assert abs(np.sum(ref_A * E) - fd) <= 1e-6 * max(abs(fd), 1.0)


def test_adjoint_unrolled_size():
    """2048 x 512, l = 16, q = 1 (the unrolled-RPCA problem size): dA entry by entry against the
    oracle's FRSVT-map adjoint."""
    fr = _fr()
    O, L, S = synth.unrolled_batch(batch=1)
    A = (O[0] - S[0]).astype(np.float32)              # rank 8 plus nothing: rank(A) <= l
    A = A + 0.01 * np.random.default_rng(3).standard_normal(A.shape).astype(np.float32)
    m, n = A.shape
    l, q, stream = 16, 1, 0
    tau = _tau_between(A, l, q, stream)
    h = fr.Handle(m, n, 16, q=q, seed=SEED, adjoint=True)
    Ad = torch.from_numpy(A).cuda()
    X, saved = h.svt_save(Ad, tau, l, stream)
    rng = np.random.default_rng(78)
    Xbar = rng.standard_normal((m, n)).astype(np.float32)
    ref_A, ref_tau, ref_X = svt.frsvt_vjp(A.astype(np.float64), tau, l, q, SEED, stream, Xbar.astype(np.float64))
    assert np.linalg.norm(X.cpu().numpy() - ref_X) <= 1e-4 * np.linalg.norm(ref_X)
    dA, dtau = h.backward(saved, Ad, tau, l, stream, torch.from_numpy(Xbar).cuda())
    torch.cuda.synchronize()
    assert h.info().device_status == 0
    _check_entrywise(dA.cpu().numpy().astype(np.float64), float(dtau.item()), ref_A, ref_tau)


def test_autograd_function_matches_backward():
    fr = _fr()
    m, n, l, q = 200, 80, 8, 1
    A = _case(m, n, 4, seed=5)
    tau = _tau_between(A, l, q, 1)
    h = fr.Handle(m, n, 16, q=q, seed=SEED, adjoint=True)
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    t = torch.tensor(tau, dtype=torch.float32, device="cuda", requires_grad=True)
    W = torch.randn(m, n, device="cuda")
    X = fr.frsvt_svt_autograd(Ad, t, h, l, 1)
    (X * W).sum().backward()
    _, saved = h.svt_save(Ad.detach(), tau, l, 1)
    dA, dtau = h.backward(saved, Ad.detach(), tau, l, 1, W)
    assert torch.allclose(Ad.grad, dA, rtol=0, atol=0)
    assert float(t.grad) == float(dtau.item())


def test_adjoint_requires_workspace_and_valid_args():
    fr = _fr()
    h = fr.Handle(100, 40, 8, q=1)
    A = torch.randn(100, 40, device="cuda")
    with pytest.raises(fr.FrsvtError):
        h.svt_save(A, 0.5, 8)
    h2 = fr.Handle(100, 40, 8, q=1, adjoint=True)
    with pytest.raises(fr.FrsvtError):
        h2.svt_save(A, -1.0, 8)
    with pytest.raises(fr.FrsvtError):
        h2.svt_save(A, 0.5, 9)                          # l > l_max
