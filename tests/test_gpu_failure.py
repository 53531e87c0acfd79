"""Failure detection on the GPU, in forms that fault, trap and hang nothing.

Every case makes the failure on the host side or with a bounded wait that is meant to run out,
then checks (1) that the call returned, (2) that the sticky device status names the failure,
and (3) that the next ordinary call on the same handle still matches the FP64 oracle:
- a NaN planted in A: the Gram reductions of the Cholesky QR report FRSVT_DEV_NONFINITE;
- a Jacobi budget of one sweep: the core SVD reports FRSVT_DEV_NOT_CONVERGED;
- a bounded mbarrier wait that nothing satisfies, with a small run-time poll limit:
  FRSVT_DEV_TIMEOUT.
"""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import svt as osvt

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


def _good_call(fr, h, m, n, l, q, seed):
    """An ordinary FRSVT on the same handle, checked against the oracle (the handle stays usable)."""
    A, s = spectrum_matrix(m, n, min(n, 3 * l), 0.9, 0.01, seed=99)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[l // 2] + s[l // 2 + 1]))
    h.reset(0)
    X = h.svt(to_gpu(A), tau, l).cpu().numpy()
    ref = osvt.frsvt(A, tau, l, q, seed=seed, stream=0)
    assert rel_fro(X, ref.X) <= TOL
    assert h.info().device_status == 0


# narrow basis on the tensor cores (n <= 256), on the CUDA cores (n > 256), wide basis (l > 32)
SHAPES = [(2000, 96, 12, 1), (1200, 300, 12, 1), (1024, 512, 64, 1)]


@pytest.mark.parametrize("m,n,l,q", SHAPES)
def test_nan_in_A_reports_nonfinite(fr, m, n, l, q):
    A, s = spectrum_matrix(m, n, min(n, 3 * l), 0.9, 0.01, seed=7)
    A = A.astype(np.float32)
    A[m // 3, n // 2] = np.nan
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5)
    h.svt(to_gpu(A), float(s[l // 2]), l)
    info = h.info()
    assert info.device_status & fr.DEV_NONFINITE, info
    _good_call(fr, h, m, n, l, q, 5)
    h.close()


def test_nan_in_O_reports_nonfinite_in_ialm(fr):
    import torch
    rng = np.random.default_rng(3)
    O = (rng.standard_normal((3000, 4)) @ rng.standard_normal((4, 120))).astype(np.float32)
    O[17, 5] = np.inf
    Og = torch.from_numpy(O).cuda()
    S, A = torch.empty_like(Og), torch.empty_like(Og)
    h = fr.Handle(3000, 120, 10, q=1, range_prop=True, seed=2)
    h.rpca_init(Og, S, A, 1.0 / np.sqrt(3000), 1.5, 1e7, normO2=50.0)
    h.ialm_step(Og, S, A, 10)
    assert h.info().device_status & fr.DEV_NONFINITE
    h.close()


@pytest.mark.parametrize("m,n,l,q", SHAPES)
def test_one_jacobi_sweep_reports_not_converged(fr, m, n, l, q):
    A, s = spectrum_matrix(m, n, min(n, 3 * l), 0.95, 0.01, seed=8)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[l // 2] + s[l // 2 + 1]))
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5, max_jacobi_sweeps=1)
    h.svt(to_gpu(A), tau, l)
    info = h.info()
    assert info.device_status & fr.DEV_NOT_CONVERGED, info
    assert info.sweeps == 1
    h.close()
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=5)           # the default budget converges
    _good_call(fr, h, m, n, l, q, 5)
    h.close()


@pytest.mark.parametrize("limit", [1, 1000, 100000])
def test_bounded_wait_runs_out(fr, limit):
    import torch
    h = fr.Handle(2000, 96, 12, q=1, range_prop=False, seed=5)
    h.debug_wait_timeout(limit)
    torch.cuda.synchronize()
    assert h.info().device_status == fr.DEV_TIMEOUT
    assert h.info().device_status == 0                              # the read cleared it
    _good_call(fr, h, 2000, 96, 12, 1, 5)
    with pytest.raises(fr.FrsvtError):
        h.debug_wait_timeout(0)
    h.close()
