"""Parity of the CUDA iALM RPCA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle import rpca as orpca
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


def run_gpu(fr, O, l, q, iters, seed, range_prop=True, orth_last=False):
    import torch
    m, n = O.shape
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    S = torch.empty_like(Og)
    A = torch.empty_like(Og)
    L = torch.empty_like(Og)
    h = fr.Handle(m, n, l, q=q, range_prop=range_prop, seed=seed, orth_last=orth_last)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(max(m, n)), 1.5, 1e7)
    hist = []
    for k in range(iters):
        hist.append(h.ialm_step(Og, S, A, l, L=L if k == iters - 1 else None, sync_residual=True))
    return L.cpu().numpy(), S.cpu().numpy(), hist, h.info()



def test_rpca_300_parity(fr):
    """300 x 300 rank 10 + 5 % corruption, l = 20, q = 1, 30 iterations, range propagation."""
    O, Ltrue, _ = synth.rpca_300()
    O32 = O.astype(np.float32).astype(np.float64)
    ref = orpca.ialm_rpca(O32, method="frsvt", l=20, q=1, seed=2001, fixed_iters=30)
    L, S, hist, info = run_gpu(fr, O32, 20, 1, 30, 2001)
    assert info.alm_iter == 30
    assert rel_fro(L, ref.L) <= TOL
    assert rel_fro(S, ref.S) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-2, atol=1e-6)
    assert rel_fro(L, Ltrue) <= 1e-4


def test_rpca_video_full_size_parity(fr):
    """76800 x 200 video-background RPCA, l = 10, q = 2, range propagation: 6 iterations."""
    O, _, _ = synth.video()
    O64 = O.astype(np.float64)
    ref = orpca.ialm_rpca(O64, method="frsvt", l=10, q=2, seed=2002, fixed_iters=6)
    L, S, hist, info = run_gpu(fr, O64, 10, 2, 6, 2002)
    assert rel_fro(L, ref.L) <= TOL
    assert rel_fro(S, ref.S) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)


def test_rpca_video_orth_last_parity(fr):
    """The video workload with the orthonormalisation only after the last power step (Sec. 2.5) on the
    tensor-core path: 6 iterations against the oracle running the same variant, and against the
    default (orthonormalise every step) oracle run."""
    O, _, _ = synth.video()
    O64 = O.astype(np.float64)
    ref = orpca.ialm_rpca(O64, method="frsvt", l=10, q=2, seed=2002, fixed_iters=6, orth_last=True)
    ref_every = orpca.ialm_rpca(O64, method="frsvt", l=10, q=2, seed=2002, fixed_iters=6)
    L, S, hist, info = run_gpu(fr, O64, 10, 2, 6, 2002, orth_last=True)
    assert rel_fro(L, ref.L) <= TOL
    assert rel_fro(S, ref.S) <= TOL
    assert rel_fro(L, ref_every.L) <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3)
