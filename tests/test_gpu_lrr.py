"""Low-rank representation (Table 6, Type A) on the GPU against the FP64 oracle `oracle/lrr.py`.

The GPU iteration (frsvt_lrr_*) runs the oracle's splitting with the J step by FRSVT (same Omega
streams, range propagation across iterations) and the L solve with a Newton-Schulz inverse of
I + Z^T Z plus one refinement step; L and S after a fixed number of iterations are compared with
the oracle's at 1e-4 relative Frobenius error, and so is the stopping quantity of every
iteration.
"""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle import lrr as olrr
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


def _run(fr, O, lam, l, q, seed, iters, mu0, rho, range_prop=True):
    import torch
    d, n = O.shape
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    h = fr.LRR(d, n, l, q=q, seed=seed, range_prop=range_prop)
    h.init(Og, lam, mu0=mu0, rho=rho)
    hist = [h.step(sync_err=True) for _ in range(iters)]
    L, S, mu, it = h.result()
    h.close()
    return L.cpu().numpy(), S.cpu().numpy(), hist, mu, it


@pytest.mark.parametrize("range_prop", [True, False])
def test_lrr_subspaces_parity(fr, range_prop):
    """synth.subspaces (60 x 60: four 3-dimensional subspaces, 10 % of the columns corrupted),
    FRSVT l = 16, q = 1, 60 iterations from mu0 = 1e-2 (rho = 1.1: mu ends near 3, so the J step
    thresholds at the scale of the iterate's singular values)."""
    O, _, _, _ = synth.subspaces()
    O = O.astype(np.float32).astype(np.float64)
    lam, K, mu0, rho = 0.25, 60, 1e-2, 1.1
    ref = olrr.lrr_ialm(O, lam, method="frsvt", l=16, q=1, seed=41, range_prop=range_prop, mu0=mu0, rho=rho,
                        fixed_iters=K)
    L, S, hist, mu, it = _run(fr, O, lam, 16, 1, 41, K, mu0, rho, range_prop)
    eL, eS = rel_fro(L, ref.L), rel_fro(S, ref.S)
    print(f"lrr 60x60 rp={range_prop}: rel err L {eL:.3e} S {eS:.3e}")
    assert it == K and abs(mu - ref.mu) <= 1e-12 * ref.mu
    assert eL <= TOL and eS <= TOL
    assert np.allclose(hist, ref.history, rtol=1e-3, atol=1e-6 * max(ref.history))


def test_lrr_wide_basis_parity(fr):
    """A larger union of subspaces (d = 200, n = 320: eight 6-dimensional subspaces, 40 columns
    each), FRSVT l = 64 (the wide basis), q = 1, 40 iterations."""
    O, _, _, _ = synth.subspaces(seed=1011, d=200, k=8, dim=6, per=40, frac=0.1)
    O = O.astype(np.float32).astype(np.float64)
    lam, K, mu0, rho = 0.3, 40, 1e-2, 1.15
    ref = olrr.lrr_ialm(O, lam, method="frsvt", l=64, q=1, seed=43, range_prop=True, mu0=mu0, rho=rho,
                        fixed_iters=K)
    L, S, hist, _, _ = _run(fr, O, lam, 64, 1, 43, K, mu0, rho)
    eL, eS = rel_fro(L, ref.L), rel_fro(S, ref.S)
    print(f"lrr 200x320 l=64: rel err L {eL:.3e} S {eS:.3e}")
    assert eL <= TOL and eS <= TOL
    # the stopping quantity is a max-norm residual, O - Z L - S or L - J: an FP32 difference of
    # entries of O's size, so the bound is 1e-3 of it plus 1e-4 of max |O|
    gap = np.abs(np.asarray(hist) - np.asarray(ref.history))
    assert np.all(gap <= 1e-3 * np.abs(ref.history) + 1e-4 * np.abs(O).max()), gap.max()


def test_lrr_invalid_arguments(fr):
    import torch
    with pytest.raises(fr.FrsvtError):
        fr.LRR(10, 1, 1)                                   # n_max < 2
    with pytest.raises(fr.FrsvtError):
        fr.LRR(10, 20, 30)                                 # l > n_max
    h = fr.LRR(10, 20, 4, q=1)
    O = torch.zeros((12, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(fr.FrsvtError):
        h.init(O, 0.1)                                     # d > d_max
    with pytest.raises(fr.FrsvtError):
        h.step()                                           # before init
    O = torch.randn((10, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(fr.FrsvtError):
        h.init(O, -1.0)                                    # lam <= 0
    h.init(O, 0.1, mu0=1e-2)
    assert np.isfinite(h.step(sync_err=True))
    h.close()
