"""Partial thresholding (Table 6, Type B, the truncated nuclear norm) on the GPU against the FP64
oracle: single FRSVT calls on both basis widths and the Type B iALM of a weather-removal window."""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import rpca as orpca
from oracle import svt as osvt
from paper_1509_00296_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


@pytest.mark.parametrize("m,n,l,q,k", [(3000, 100, 16, 2, 2), (20000, 200, 10, 1, 1), (2048, 1024, 64, 2, 3)])
def test_partial_frsvt_matches_oracle(fr, m, n, l, q, k):
    A, s = spectrum_matrix(m, n, l + 8, 0.85, 0.01, seed=7 * m + n)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[k + 2] + s[k + 3]))
    ref = osvt.frsvt(A, tau, l, q, seed=3, stream=0, partial_k=k)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=3)
    h.set_partial(k)
    X = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    info = h.info()
    h.close()
    assert info.r == ref.r
    assert rel_fro(X, ref.X) <= TOL


def test_type_b_ialm_weather_window(fr):
    """One 5-frame window of the snow video (110592 x 5), Type B iALM with k = 1, l = 3, q = 2 and
    range propagation (the weather-removal settings), 30 iterations against the oracle."""
    import torch
    O, clean, mask = synth.snow_video(frames=5)
    O64 = O.astype(np.float64)
    ref = orpca.ialm_rpca(O64, method="frsvt", l=3, q=2, seed=8, partial_k=1, fixed_iters=30)
    m, n = O.shape

    def padded():                                   # leading dimension 8 (TMA rows: multiples of 16 bytes)
        return torch.zeros((m, 8), dtype=torch.float32, device="cuda")[:, :n]

    Og, S, A, L = padded(), padded(), padded(), padded()
    Og.copy_(torch.from_numpy(O))
    h = fr.Handle(m, n, 3, q=2, range_prop=True, seed=8)
    h.set_partial(1)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(m), 1.5, 1e7)
    for k in range(30):
        h.ialm_step(Og, S, A, 3, L=L if k == 29 else None, sync_residual=True)
    h.close()
    Lh, Sh = L.cpu().numpy(), S.cpu().numpy()
    assert rel_fro(Lh, ref.L) <= TOL
    assert rel_fro(Sh, ref.S) <= TOL
    # the snow is in S: most flake pixels carry a clearly positive sparse part
    assert np.mean(Sh[mask] > 0.05) > 0.9
