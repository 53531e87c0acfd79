"""Parity of the CUDA FRSVT path (through the C ABI) with the FP64 oracle.

Tolerance: relative Frobenius error <= 1e-4 between the FP32 GPU result and the
FP64 oracle on the same input (cast to FP32) and the same Omega stream.
"""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import philox, svt

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


def test_philox_words_bit_exact(fr):
    for seed, stream, prob in ((0, 0, 0), (2001, 7, 0), (2**63 + 5, 2**40 + 3, 9)):
        got = fr.debug_philox(777, 5, seed, stream, prob).cpu().numpy().view(np.uint64)
        ref = philox.philox_words(777, 20, seed, stream, prob)
        assert np.array_equal(got, ref)


def test_omega_matches_oracle(fr):
    for rows, cols, seed, stream in ((5000, 13, 3, 1), (1000, 32, 2002, 0), (7, 1, 1, 5)):
        got = fr.debug_omega(rows, cols, seed, stream).cpu().numpy()
        ref = philox.gaussian_matrix(rows, cols, seed, stream)
        assert np.max(np.abs(got - ref)) < 3e-5
        assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) < 1e-5


CASES = [  # m, n, rank, decay, noise, l, q, ld
    (300, 300, 40, 0.85, 0.01, 20, 1, None),
    (1000, 64, 30, 0.8, 0.001, 10, 2, None),
    (2049, 77, 30, 0.8, 0.001, 12, 0, 80),        # ragged rows and columns, padded leading dimension
    (513, 200, 60, 0.9, 0.01, 16, 2, None),
    (700, 300, 60, 0.93, 0.01, 32, 1, 304),
    (4100, 33, 20, 0.7, 0.0, 5, 1, 36),
    (3000, 1500, 60, 0.9, 0.01, 16, 1, None),     # short side too wide for the fused single-CTA tails
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}_l{c[5]}_q{c[6]}" for c in CASES])
def test_frsvt_matches_oracle(fr, case):
    m, n, rank, decay, noise, l, q, ld = case
    A, s = spectrum_matrix(m, n, rank, decay, noise, seed=m + n)
    A = A.astype(np.float32).astype(np.float64)
    k = l // 2
    tau = float(0.5 * (s[k - 1] + s[k]))
    ref = svt.frsvt(A, tau, l, q, seed=11, stream=0)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=11)
    Ag = to_gpu(A, ld)
    X = h.svt(Ag, tau, l, X=to_gpu(np.zeros((m, n)), ld)).cpu().numpy()
    info = h.info()
    assert info.r == ref.r
    assert info.device_status & fr.DEV_NONFINITE == 0
    assert rel_fro(X, ref.X) <= TOL
    sig = np.array(h.sigma())
    assert np.max(np.abs(sig[: ref.r] - ref.sigma[: ref.r])) <= 1e-4 * ref.sigma[0]


def test_frsvt_exact_for_low_rank(fr):
    """rank(A) <= l: FRSVT equals the exact SVT (remark after Cor. 2)."""
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((3000, 5)) @ rng.standard_normal((5, 120))).astype(np.float32).astype(np.float64)
    sv = np.linalg.svd(A, compute_uv=False)
    tau = float(0.5 * (sv[2] + sv[3]))
    Xe, r = svt.exact_svt(A, tau)
    h = fr.Handle(3000, 120, 10, q=1, range_prop=False, seed=3)
    X = h.svt(to_gpu(A), tau, 10).cpu().numpy()
    assert h.info().r == r == 3
    assert rel_fro(X, Xe) <= TOL


@pytest.mark.parametrize("m,n", [(1500, 120), (1500, 300)])
def test_frsvt_range_propagation_sequence(fr, m, n):
    """Three calls on a slowly moving iterate: the propagated basis (Alg. 1 steps 8-11) matches the oracle,
    and so does the Prop. 4 residual ||(I - Q~ Q~^T) A^T omega_0|| of the first new sample column
    (n = 120: tensor-core sketch tail; n = 300: CUDA-core path)."""
    l, q = 12, 1
    A0, s = spectrum_matrix(m, n, 30, 0.75, 0.001, seed=77)
    rng = np.random.default_rng(78)
    Dlt = rng.standard_normal((m, n)) * 0.01
    tau = float(0.5 * (s[5] + s[6]))
    h = fr.Handle(m, n, l, q=q, range_prop=True, seed=21)
    Qp = None
    for t in range(3):
        A = (A0 + t * Dlt).astype(np.float32).astype(np.float64)
        kept = 0 if Qp is None else Qp.shape[1]
        ref = svt.frsvt(A, tau, l, q, seed=21, stream=t, Q_prev=Qp)
        Qp = ref.Q_tilde
        X = h.svt(to_gpu(A), tau, l).cpu().numpy()
        info = h.info()
        assert info.r == ref.r and info.keep == ref.Q_tilde.shape[1]
        assert info.counter == t + 1
        assert rel_fro(X, ref.X) <= TOL, t
        want = ref.extra["rp_residual"]
        if kept == 0:
            assert want == -1.0 and info.rp_residual == -1.0 and info.residual_estimate() == -1.0, t
        else:
            # a difference of FP32 quantities of size ||y||: 1e-3 of the residual plus 1e-5 ||y||
            y = A.T @ philox.gaussian_matrix(m, l - kept, 21, t, 0)[:, 0]
            assert abs(info.rp_residual - want) <= 1e-3 * want + 1e-5 * np.linalg.norm(y), (t, info.rp_residual, want)


@pytest.mark.parametrize("q", [2, 3])
def test_frsvt_orth_last_matches_oracle(fr, q):
    """FRSVT_CFG_ORTH_LAST (Sec. 2.5): the tensor-core path skips the orthonormalisation of the
    intermediate power steps; X matches the oracle running the same variant, over a range-propagated
    sequence of two calls."""
    m, n, l = 3000, 200, 12
    A, s = spectrum_matrix(m, n, 40, 0.85, 0.001, seed=91)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[6] + s[7]))
    h = fr.Handle(m, n, l, q=q, range_prop=True, seed=31, orth_last=True)
    Qp = None
    for t in range(2):
        ref = svt.frsvt(A, tau, l, q, seed=31, stream=t, Q_prev=Qp, orth_last=True)
        Qp = ref.Q_tilde
        X = h.svt(to_gpu(A), tau, l).cpu().numpy()
        info = h.info()
        assert info.r == ref.r, t
        assert rel_fro(X, ref.X) <= TOL, t


def test_tau_above_sigma_max_gives_zero(fr):
    A, s = spectrum_matrix(400, 50, 10, 0.8, 0.0, seed=9)
    h = fr.Handle(400, 50, 8, q=1, range_prop=False)
    X = h.svt(to_gpu(A), float(2 * s[0]), 8, X=to_gpu(np.full((400, 50), 7.0))).cpu().numpy()
    assert np.all(X == 0.0)
    assert h.info().r == 0


def test_tau_zero_full_basis_returns_input(fr):
    """l >= n and tau = 0: Q spans everything and S_0(A) = A."""
    rng = np.random.default_rng(10)
    A = rng.standard_normal((900, 12)).astype(np.float32)
    h = fr.Handle(900, 12, 16, q=1, range_prop=False)
    X = h.svt(to_gpu(A), 0.0, 16).cpu().numpy()
    assert rel_fro(X, A) <= 1e-5


def test_spectral_norm(fr):
    A, s = spectrum_matrix(2000, 150, 40, 0.9, 0.01, seed=12)
    h = fr.Handle(2000, 150, 16, q=1)
    assert abs(h.spectral_norm(to_gpu(A), 20) - np.linalg.norm(A, 2)) <= 1e-5 * np.linalg.norm(A, 2)


def test_invalid_arguments(fr):
    import torch
    h = fr.Handle(256, 64, 8, q=1)
    A = torch.zeros((256, 64), device="cuda")
    with pytest.raises(fr.FrsvtError) as e:
        h.svt(A.t().contiguous(), 1.0, 8)                  # 64 x 256: m < n
    assert e.value.status == 2
    big = torch.zeros((256, 68), device="cuda")
    with pytest.raises(fr.FrsvtError) as e:
        h.svt(big[:, 1:65], 1.0, 8)                        # base not 16-byte aligned
    assert e.value.status == 1
    with pytest.raises(fr.FrsvtError) as e:
        h.svt(torch.zeros((300, 64), device="cuda"), 1.0, 8)   # larger than m_max
    assert e.value.status == 1
    with pytest.raises(fr.FrsvtError) as e:
        h.svt(A, 1.0, 9)                                    # l > l_max
    assert e.value.status == 1
    odd = torch.zeros((256, 66), device="cuda")[:, :64]     # leading dimension 66 is not a multiple of 4
    with pytest.raises(fr.FrsvtError) as e:
        h.svt(odd, 1.0, 8)
    assert e.value.status == 1
    empty = torch.zeros((0, 0), device="cuda")
    h.svt(empty, 1.0, 8)                                    # empty problem: a no-op
