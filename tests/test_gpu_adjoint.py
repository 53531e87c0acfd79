"""Adjoint of the FRSVT map (frsvt_svt_save / frsvt_backward) against the FP64 oracle.

The FRSVT map with a fixed Omega is differentiated; the oracle differentiates its own FP64
FRSVT with the same Omega by central differences (h = 1e-3) along random directions, taken
where no singular value of B sits near tau.  The exact-SVD gradient is reported beside it.
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


@pytest.mark.parametrize("shape,l,q", [((300, 120), 8, 1), ((257, 96), 12, 2)])
def test_adjoint_matches_oracle_fd(shape, l, q):
    fr = _fr()
    m, n = shape
    A = _case(m, n, 5, seed=31 + m)
    stream = 3
    tau = _tau_between(A, l, q, stream)
    h = fr.Handle(m, n, 16, q=q, seed=SEED, adjoint=True)
    Ad = torch.from_numpy(A).cuda()
    X, saved = h.svt_save(Ad, tau, l, stream)
    torch.cuda.synchronize()
    ref = svt.frsvt(A.astype(np.float64), tau, l, q, SEED, stream).X
    assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
    rng = np.random.default_rng(77)
    Xbar = rng.standard_normal((m, n)).astype(np.float32)
    dA, dtau = h.backward(saved, Ad, tau, l, stream, torch.from_numpy(Xbar).cuda())
    torch.cuda.synchronize()
    assert h.info().device_status & (fr.DEV_RANK_DEFICIENT | fr.DEV_NONFINITE) == 0
    dA = dA.cpu().numpy().astype(np.float64)
    for k in range(4):
        E = rng.standard_normal((m, n))
        fd = svt.frsvt_directional_fd(A.astype(np.float64), tau, l, q, SEED, stream, Xbar.astype(np.float64), E)
        got = float(np.sum(dA * E))
        assert abs(got - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.linalg.norm(dA) * np.linalg.norm(E)), (k, got, fd)
    fdt = svt.frsvt_directional_fd(A.astype(np.float64), tau, l, q, SEED, stream, Xbar.astype(np.float64),
                                   np.zeros((m, n)), dtau=1.0)
    assert abs(float(dtau.item()) - fdt) <= 1e-3 * max(abs(fdt), 1.0)
    if shape == (300, 120):
        Ae, te = svt.svt_vjp(A.astype(np.float64), tau, Xbar.astype(np.float64))
        gap = np.linalg.norm(dA - Ae) / np.linalg.norm(Ae)
        print(f"relative gap to the exact-SVD gradient: {gap:.3e} (dtau {float(dtau.item()):.4g} vs {te:.4g})")
        assert np.isfinite(gap)


def test_adjoint_unrolled_size():
    """2048 x 512, l = 16, q = 1 (the unrolled-RPCA problem size): FD along two directions."""
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
    ref = svt.frsvt(A.astype(np.float64), tau, l, q, SEED, stream).X
    assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
    rng = np.random.default_rng(78)
    Xbar = rng.standard_normal((m, n)).astype(np.float32)
    dA, dtau = h.backward(saved, Ad, tau, l, stream, torch.from_numpy(Xbar).cuda())
    dA = dA.cpu().numpy().astype(np.float64)
    for k in range(2):
        E = rng.standard_normal((m, n))
        fd = svt.frsvt_directional_fd(A.astype(np.float64), tau, l, q, SEED, stream, Xbar.astype(np.float64), E)
        got = float(np.sum(dA * E))
        assert abs(got - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.linalg.norm(dA) * np.linalg.norm(E)), (k, got, fd)


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
