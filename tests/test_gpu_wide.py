"""Parity of the wide-basis path (32 < l <= 128, any short side) with the FP64 oracle.

The large low-rank recovery configuration runs FRSVT with l = 120 on an 8192 x 8192 matrix;
the basis then spans several 256-column tiles of the tensor-core passes and the small dense
steps (Cholesky QR, the l x l core) run as grid-wide kernels.  Parity is checked on shapes that
span several tiles with ragged tails, on a rank-deficient input, on iALM iterations, and on the
full-size configuration.
"""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import rpca as orpca
from oracle import svt as osvt
from paper_1509_00296_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
FP8_TOL = 1e-3


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


def power_norm2(O, iters=40, seed=0):
    """||O||_2 estimate (FP64 power method); both sides receive the same value."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(O.shape[1])
    s = 0.0
    for _ in range(iters):
        u = O @ v
        v = O.T @ u
        s = np.linalg.norm(v)
        v /= s
    return float(np.sqrt(s))


@pytest.mark.parametrize("m,n,l,q,rank,decay", [
    (1000, 700, 120, 2, 160, 0.985),
    (2048, 2048, 120, 1, 200, 0.99),
    (777, 333, 50, 1, 80, 0.97),
    (600, 90, 48, 2, 60, 0.95),
    (1500, 1000, 96, 0, 110, 0.98),
    (900, 400, 37, 1, 50, 0.96),
])
def test_wide_frsvt_parity(fr, m, n, l, q, rank, decay):
    """FRSVT with a wide basis: X, r and the leading sigma against the oracle's Alg. 1."""
    A, s = spectrum_matrix(m, n, rank, decay, 0.01, seed=31 * m + n)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[l // 2] + s[l // 2 + 1]))
    ref = osvt.frsvt(A, tau, l, q, seed=11, stream=0)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=11)
    X = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    assert info.device_status == 0, info          # full-rank, well-separated spectrum: s = l
    assert info.s == min(l, n)
    assert rel_fro(X, ref.X) <= TOL
    assert info.r == ref.r
    sig = h.sigma()
    k = ref.r
    assert np.allclose(sig[:k], ref.sigma[:k], rtol=1e-4)
    h.close()


def test_wide_rank_deficient(fr):
    """rank(A) = 20 < l = 64: X equals the exact SVT; the rank cut keeps the basis usable."""
    m, n = 1200, 900
    A, s = spectrum_matrix(m, n, 20, 0.9, 0.0, seed=5)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[9] + s[10]))
    ref, _ = osvt.exact_svt(A, tau)
    h = fr.Handle(m, n, 64, q=1, range_prop=False, seed=3)
    X = h.svt(to_gpu(A), tau, 64, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    # rank 20 < l: the Cholesky QR drops the surplus columns and says so (informational bit)
    assert info.device_status == fr.DEV_RANK_DEFICIENT, info
    assert 20 <= info.s < 64, info
    assert rel_fro(X, ref) <= TOL
    assert info.r == 10
    h.close()


def test_wide_ragged_leading_dimension(fr):
    """Padded rows (ld > n) and sizes that are not multiples of any tile."""
    m, n, l = 1031, 517, 72
    A, s = spectrum_matrix(m, n, 90, 0.97, 0.01, seed=9)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[30] + s[31]))
    ref = osvt.frsvt(A, tau, l, 1, seed=4, stream=0)
    h = fr.Handle(m, n, l, q=1, range_prop=False, seed=4)
    ld = n + 7 + 4 - (n + 7) % 4
    X = h.svt(to_gpu(A, ld=ld), tau, l, X=to_gpu(np.zeros_like(A), ld=ld)).cpu().numpy()
    assert rel_fro(X, ref.X) <= TOL
    h.close()


def run_ialm(fr, O, l, q, iters, seed, normO2):
    import torch
    m, n = O.shape
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S, A, L = torch.empty_like(Og), torch.empty_like(Og), torch.empty_like(Og)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=seed)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7, normO2=normO2)
    hist = []
    for k in range(iters):
        hist.append(h.ialm_step(Og, S, A, l, L=L if k == iters - 1 else None, sync_residual=True))
    info = h.info()
    out = L.cpu().numpy(), S.cpu().numpy(), hist, info
    h.close()
    return out


def test_wide_ialm_parity(fr):
    """iALM with FRSVT (l = 60, q = 2) on 1024 x 1024 rank 20 + 10 % corruption: 4 iterations."""
    O, _, _ = synth.lowrank_sparse(1024, 1024, 20, 0.10, 10.0, seed=77, scale=1.0 / np.sqrt(20.0))
    O = O.astype(np.float32).astype(np.float64)
    nrm = power_norm2(O)
    ref = orpca.ialm_rpca(O, method="frsvt", l=60, q=2, seed=2003, range_prop=False, fixed_iters=4, normO2=nrm)
    L, S, hist, info = run_ialm(fr, O, 60, 2, 4, 2003, nrm)
    assert info.alm_iter == 4
    assert rel_fro(L, ref.L) <= TOL
    assert rel_fro(S, ref.S) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)


@pytest.fixture(scope="module")
def recovery_ref():
    """Oracle iALM-FRSVT on the large low-rank recovery input (three iterations, FP64)."""
    O, _, _ = synth.recovery_8192()
    O = O.astype(np.float64)
    nrm = power_norm2(O, iters=30)
    ref = orpca.ialm_rpca(O, method="frsvt", l=120, q=2, seed=2004, range_prop=False, fixed_iters=3, normO2=nrm)
    return O, nrm, ref


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_wide_recovery_8192_full_size(fr, recovery_ref, prec):
    """Large low-rank recovery, 8192 x 8192 rank 100 + 10 % corruption, FRSVT l = 120, q = 2:
    three iALM iterations at full size against the oracle, FP32-accurate passes and the BF16
    shadow (sketch and first power step in BF16, FP32-accurate last power step and projection)."""
    import torch
    O, nrm, ref = recovery_ref
    m, n = O.shape
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S, A, L = torch.empty_like(Og), torch.empty_like(Og), torch.empty_like(Og)
    h = fr.Handle(m, n, 120, q=2, range_prop=False, seed=2004,
                  precision={"fp32": fr.PREC_FP32, "bf16": fr.PREC_BF16, "fp8": fr.PREC_FP8}[prec])
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7, normO2=nrm)
    hist = [h.ialm_step(Og, S, A, 120, L=L if k == 2 else None, sync_residual=True) for k in range(3)]
    info = h.info()
    h.close()
    eL = rel_fro(L.cpu().numpy(), ref.L)
    eS = rel_fro(S.cpu().numpy(), ref.S)
    print(f"recovery 8192 {prec}: rel err L {eL:.3e} S {eS:.3e}")
    # the first iterations' iterates are full rank at l = 120 (the tail singular values shrink like
    # 1 / mu and reach the rank cut only after ~18 iterations), so no column may be dropped here
    assert info.device_status == 0, info
    tol = FP8_TOL if prec == "fp8" else TOL
    assert eL <= tol
    assert eS <= tol
    assert np.allclose(hist, ref.history, rtol=1e-3 if prec != "fp8" else 1e-2)


@pytest.mark.parametrize("variant", ["range_prop", "orth_last"])
def test_wide_recovery_8192_variants(fr, recovery_ref, variant):
    """The large low-rank recovery with range propagation (Alg. 1 steps 8-11: each iteration
    sketches l - keep new columns next to the previous iteration's Q~) or with the intermediate
    power step left unnormalised (Sec. 2.5): three iALM iterations at full size against the oracle
    running the same variant."""
    import torch
    O, nrm, _ = recovery_ref
    m, n = O.shape
    rp, ol = variant == "range_prop", variant == "orth_last"
    ref = orpca.ialm_rpca(O, method="frsvt", l=120, q=2, seed=2004, range_prop=rp, orth_last=ol, fixed_iters=3,
                          normO2=nrm)
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S, A, L = torch.empty_like(Og), torch.empty_like(Og), torch.empty_like(Og)
    h = fr.Handle(m, n, 120, q=2, range_prop=rp, seed=2004, orth_last=ol)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7, normO2=nrm)
    hist = [h.ialm_step(Og, S, A, 120, L=L if k == 2 else None, sync_residual=True) for k in range(3)]
    info = h.info()
    h.close()
    eL = rel_fro(L.cpu().numpy(), ref.L)
    eS = rel_fro(S.cpu().numpy(), ref.S)
    print(f"recovery 8192 {variant}: rel err L {eL:.3e} S {eS:.3e}, keep {info.keep}")
    assert info.device_status == 0, info
    if rp:
        assert info.keep == min(info.r, 118) and info.keep > 0
    assert eL <= TOL
    assert eS <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)


@pytest.mark.parametrize("m,n", [(2048, 1024), (1024, 2048)])
def test_wide_range_propagation_sequence(fr, m, n):
    """Range propagation on the wide basis, both orientations: three calls on a slowly moving
    iterate, each X against the oracle given the previous oracle call's Q~ (keep = min(r, l - 2)
    columns carried over, on the short side)."""
    l, q = 64, 1
    A0, s = spectrum_matrix(m, n, 80, 0.95, 0.001, seed=201)
    rng = np.random.default_rng(202)
    D = rng.standard_normal((m, n)) * 0.01
    tau = float(0.5 * (s[30] + s[31]))
    h = fr.Handle(max(m, n), max(m, n), l, q=q, range_prop=True, seed=23)
    Qp = None
    for t in range(3):
        A = (A0 + t * D).astype(np.float32).astype(np.float64)
        ref = osvt.frsvt(A, tau, l, q, seed=23, stream=t, Q_prev=Qp)
        Qp = ref.Q_tilde
        X = h.svt(to_gpu(A), tau, l).cpu().numpy()
        info = h.info()
        assert info.r == ref.r and info.keep == ref.Q_tilde.shape[1], (t, info.r, ref.r, info.keep)
        assert info.counter == t + 1
        assert info.rp_residual == -1.0                 # the wide basis computes no Prop. 4 residual
        assert rel_fro(X, ref.X) <= TOL, t
    h.close()


@pytest.mark.parametrize("q", [2, 3])
def test_wide_orth_last_matches_oracle(fr, q):
    """FRSVT_CFG_ORTH_LAST on the wide basis: the intermediate power steps are not orthonormalised;
    X matches the oracle's same variant over a range-propagated sequence of two calls."""
    m, n, l = 2048, 1024, 64
    A, s = spectrum_matrix(m, n, 80, 0.95, 0.001, seed=211)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[20] + s[21]))
    h = fr.Handle(m, n, l, q=q, range_prop=True, seed=37, orth_last=True)
    Qp = None
    for t in range(2):
        ref = osvt.frsvt(A, tau, l, q, seed=37, stream=t, Q_prev=Qp, orth_last=True)
        Qp = ref.Q_tilde
        X = h.svt(to_gpu(A), tau, l).cpu().numpy()
        assert h.info().r == ref.r, t
        assert rel_fro(X, ref.X) <= TOL, t
    h.close()


@pytest.mark.parametrize("m,n,l,q", [(2048, 1024, 64, 2), (1500, 700, 120, 2), (1200, 600, 40, 3)])
def test_wide_bf16_svt_matches_oracle(fr, m, n, l, q):
    """BF16 shadow on the wide basis: X against the oracle's FP32-free Alg. 1 at the 1e-4 bar."""
    A, _ = spectrum_matrix(m, n, rank=l + 8, decay=0.93, noise=0.01, seed=m + 3 * n)
    d = osvt.frsvt(A.astype(np.float64), 0.0, l, q, 5, 0).sigma
    tau = float(0.5 * (d[l // 3] + d[l // 3 + 1]))
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5, precision=fr.PREC_BF16)
    X = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    assert info.device_status & (fr.DEV_TIMEOUT | fr.DEV_NONFINITE) == 0
    ref = osvt.frsvt(A.astype(np.float64), tau, l, q, 5, 0).X
    assert rel_fro(X, ref) <= TOL
    h.close()


@pytest.mark.parametrize("m,n,l,q", [(2048, 1024, 64, 2), (1500, 700, 120, 2), (1200, 600, 40, 3)])
def test_wide_fp8_svt_against_oracle(fr, m, n, l, q):
    """E4M3 shadow with per-128 x 128-tile power-of-two scales for the sketch and the early power
    steps: X against the oracle (error reported; FP32-accurate last power step and projection)."""
    A, _ = spectrum_matrix(m, n, rank=l + 8, decay=0.93, noise=0.01, seed=m + 3 * n)
    d = osvt.frsvt(A.astype(np.float64), 0.0, l, q, 5, 0).sigma
    tau = float(0.5 * (d[l // 3] + d[l // 3 + 1]))
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5, precision=fr.PREC_FP8)
    X = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    assert info.device_status & (fr.DEV_TIMEOUT | fr.DEV_NONFINITE | fr.DEV_BAD_PROBLEM) == 0
    ref = osvt.frsvt(A.astype(np.float64), tau, l, q, 5, 0).X
    err = rel_fro(X, ref)
    print(f"fp8 svt {m}x{n} l={l} q={q}: rel err {err:.3e}")
    assert err <= FP8_TOL
    h.close()


def test_fp8_needs_wide_basis(fr):
    with pytest.raises(fr.FrsvtError):
        fr.Handle(100, 40, 16, q=1, precision=fr.PREC_FP8)


def test_wide_edges(fr):
    """Edge cases of the wide basis: empty input, the largest basis (l = 128), l clamped to a
    short side below l, and the m < n rejection."""
    import torch
    h = fr.Handle(1024, 512, 128, q=1, range_prop=False, seed=9)
    empty = torch.zeros((8, 0), dtype=torch.float32, device="cuda")
    h.svt(empty, 1.0, 64, X=torch.zeros_like(empty))                 # nothing to do, no error
    A, s = spectrum_matrix(1024, 512, 160, 0.985, 0.01, seed=13)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[60] + s[61]))
    X = h.svt(to_gpu(A), tau, 128).cpu().numpy()
    ref = osvt.frsvt(A, tau, 128, 1, seed=9, stream=0)
    assert rel_fro(X, ref.X) <= TOL
    W = np.ascontiguousarray(A[:100, :200])                          # m < n: the passes swap roles
    Xw = h.svt(to_gpu(W), tau / 4, 64).cpu().numpy()
    refw = osvt.frsvt(W, tau / 4, 64, 1, seed=9, stream=1)
    assert rel_fro(Xw, refw.X) <= TOL
    h.close()
    hn = fr.Handle(200, 200, 16, q=1, range_prop=False, seed=9)        # the narrow basis stays tall-only
    with pytest.raises(fr.FrsvtError):
        hn.svt(to_gpu(W), tau, 8)
    hn.close()
    # l (100) above the short side (60): clamped to 60 on both sides
    B, sb = spectrum_matrix(600, 60, 40, 0.9, 0.01, seed=17)
    B = B.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (sb[10] + sb[11]))
    h = fr.Handle(600, 60, 100, q=2, range_prop=False, seed=2)
    X = h.svt(to_gpu(B), tau, 100).cpu().numpy()
    ref = osvt.frsvt(B, tau, 100, 2, seed=2, stream=0)
    assert rel_fro(X, ref.X) <= TOL
    h.close()


@pytest.mark.parametrize("m,n,l,q", [(700, 2048, 60, 2), (333, 1031, 37, 1), (1000, 1001, 96, 0)])
def test_wide_basis_serves_m_less_than_n(fr, m, n, l, q):
    """m < n: the basis lives on the row side, Omega has n rows; X, r, sigma and the factored form
    against the oracle's Alg. 1 (which takes the same orientation)."""
    A, s = spectrum_matrix(m, n, min(m, l + 40), 0.97, 0.01, seed=7 * m + n)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[l // 2] + s[l // 2 + 1]))
    ref = osvt.frsvt(A, tau, l, q, seed=23, stream=0)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=23)
    X = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    assert info.device_status == 0, info
    assert rel_fro(X, ref.X) <= TOL
    assert info.r == ref.r
    assert np.allclose(h.sigma()[:ref.r], ref.sigma[:ref.r], rtol=1e-4)
    ref1 = osvt.frsvt(A, tau, l, q, seed=23, stream=1)
    U, V, r = h.svt_factors(to_gpu(A), tau, l)
    assert rel_fro((U.double() @ V.double().T).cpu().numpy(), ref1.X) <= TOL
    assert int(r.item()) == ref1.r
    h.close()


def test_wide_ialm_ragged_columns(fr):
    """iALM on 1031 x 517 (neither side a multiple of 4 or of a tile) stored with ld = 520: the
    fused epilogue's last column group reads one float of each row and zero-fills the rest;
    4 iterations against the oracle."""
    import torch
    O, _, _ = synth.lowrank_sparse(1031, 517, 12, 0.10, 10.0, seed=79, scale=1.0 / np.sqrt(12.0))
    O = O.astype(np.float32).astype(np.float64)
    m, n, l, iters = 1031, 517, 40, 4
    nrm = power_norm2(O)
    ref = orpca.ialm_rpca(O, method="frsvt", l=l, q=1, seed=2006, range_prop=False, fixed_iters=iters, normO2=nrm)
    Og = to_gpu(O, ld=520)
    S, A, L = to_gpu(np.zeros_like(O), ld=520), to_gpu(np.zeros_like(O), ld=520), to_gpu(np.zeros_like(O), ld=520)
    h = fr.Handle(m, n, l, q=1, range_prop=False, seed=2006)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7, normO2=nrm)
    hist = [h.ialm_step(Og, S, A, l, L=L if k == iters - 1 else None, sync_residual=True) for k in range(iters)]
    info = h.info()
    h.close()
    assert info.alm_iter == iters and info.device_status == 0, info
    assert rel_fro(L.cpu().numpy(), ref.L) <= TOL
    assert rel_fro(S.cpu().numpy(), ref.S) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)
    Sp = S.as_strided((m, 520), (520, 1)).cpu().numpy()
    assert np.all(Sp[:, n:] == 0.0)                                  # the padding is never written


def test_wide_ialm_m_less_than_n(fr):
    """iALM on a wide O (512 x 1500, rank 20 + 10 % corruption): 4 iterations against the oracle."""
    O, _, _ = synth.lowrank_sparse(512, 1500, 20, 0.10, 10.0, seed=78, scale=1.0 / np.sqrt(20.0))
    O = O.astype(np.float32).astype(np.float64)
    nrm = power_norm2(O)
    ref = orpca.ialm_rpca(O, method="frsvt", l=60, q=2, seed=2005, range_prop=False, fixed_iters=4, normO2=nrm)
    L, S, hist, info = run_ialm(fr, O, 60, 2, 4, 2005, nrm)
    assert info.alm_iter == 4 and info.device_status == 0, info
    assert rel_fro(L, ref.L) <= TOL
    assert rel_fro(S, ref.S) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)


def test_wide_recovery_8192_twenty_iterations(fr, recovery_ref):
    """The headline workload at bench length: 20 iALM iterations of the 8192 x 8192 recovery (FRSVT
    l = 120, q = 2) against the FP64 oracle, L and S at 1e-4 and the residual history at 1e-3.  From
    about the 18th iteration the iterate is numerically rank 100 and the Cholesky QR may drop basis
    columns whose singular values lie far below tau (the informational rank bit); X is unaffected."""
    import torch
    O, nrm, _ = recovery_ref
    m, n = O.shape
    iters = 20
    ref = orpca.ialm_rpca(O, method="frsvt", l=120, q=2, seed=2004, range_prop=False, fixed_iters=iters,
                          normO2=nrm)
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S, A, L = torch.empty_like(Og), torch.empty_like(Og), torch.empty_like(Og)
    h = fr.Handle(m, n, 120, q=2, range_prop=False, seed=2004)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7, normO2=nrm)
    hist = [h.ialm_step(Og, S, A, 120, L=L if k == iters - 1 else None, sync_residual=True) for k in range(iters)]
    info = h.info()
    h.close()
    eL = rel_fro(L.cpu().numpy(), ref.L)
    eS = rel_fro(S.cpu().numpy(), ref.S)
    print(f"recovery 8192, {iters} iterations: rel err L {eL:.3e} S {eS:.3e}")
    assert info.alm_iter == iters
    assert info.device_status & ~fr.DEV_RANK_DEFICIENT == 0, info
    assert eL <= TOL
    assert eS <= TOL
    # late residuals (~1e-5 of ||O||) are of the order of the allowed L and S differences themselves,
    # so the history is compared at 1e-3 relative or the parity bar absolute
    assert np.allclose(hist, ref.history, rtol=1e-3, atol=TOL)
