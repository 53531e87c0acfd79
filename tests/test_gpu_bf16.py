"""Reduced precision (BF16 shadow of A for the sketch and the early power steps, FP32-accurate
last power step and projection) against the FP64 oracle, at the 1e-4 bar of the FP32 path."""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import rpca as orpca
from oracle import svt
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


@pytest.mark.parametrize("m,n,l,q", [(3000, 128, 16, 2), (20000, 200, 10, 2), (5000, 96, 12, 1)])
def test_bf16_svt_matches_oracle(fr, m, n, l, q):
    A, _ = spectrum_matrix(m, n, rank=l + 8, decay=0.7, noise=0.01, seed=m + n)
    d = svt.frsvt(A.astype(np.float64), 0.0, l, q, 5, 0).sigma
    tau = float(0.5 * (d[2] + d[3]))
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5, precision=fr.PREC_BF16)
    Ad = to_gpu(A)
    X = h.svt(Ad, tau, l)
    info = h.info()
    assert info.device_status & (fr.DEV_TIMEOUT | fr.DEV_NONFINITE) == 0
    ref = svt.frsvt(A.astype(np.float64), tau, l, q, 5, 0).X
    assert rel_fro(X.cpu().numpy(), ref) <= TOL


def test_bf16_unsupported_precision_value(fr):
    with pytest.raises(fr.FrsvtError):
        fr.Handle(100, 40, 8, q=1, precision=7)


def test_bf16_rpca_video_full_size(fr):
    """76800 x 200 video-background RPCA, l = 10, q = 2, range propagation, 6 iterations in BF16 mode."""
    import torch
    O, _, _ = synth.video()
    O64 = O.astype(np.float64)
    ref = orpca.ialm_rpca(O64, method="frsvt", l=10, q=2, seed=2002, fixed_iters=6)
    m, n = O.shape
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S = torch.empty_like(Og)
    A = torch.empty_like(Og)
    L = torch.empty_like(Og)
    h = fr.Handle(m, n, 10, q=2, range_prop=True, seed=2002, precision=fr.PREC_BF16)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7)
    for k in range(6):
        h.ialm_step(Og, S, A, 10, L=L if k == 5 else None, sync_residual=True)
    assert rel_fro(L.cpu().numpy(), ref.L) <= TOL
    assert rel_fro(S.cpu().numpy(), ref.S) <= TOL
