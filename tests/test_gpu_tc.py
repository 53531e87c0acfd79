"""The tensor-core (tcgen05, 3xTF32) row pass Z = A Q against the exact FP64 product."""
import numpy as np
import pytest

from gpu_util import to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


@pytest.mark.parametrize("m,n,LP", [(5000, 200, 16), (1000, 256, 16), (777, 77, 16), (300, 32, 16),
                                    (4100, 200, 32), (129, 5, 16)])
def test_rows_tc_matches_fp64(fr, m, n, LP):
    import torch
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    Q = rng.standard_normal((n, LP)).astype(np.float32)
    h = fr.Handle(m, n, LP, q=1)
    Z = h.debug_rows_tc(to_gpu(A), torch.from_numpy(Q).cuda()).cpu().numpy()
    ref = A.astype(np.float64) @ Q.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(Q).astype(np.float64)   # error bound of a dot product
    err = np.max(np.abs(Z - ref) / scale)
    assert h.info().device_status & fr.DEV_NONFINITE == 0
    assert err < 2e-6, err


@pytest.mark.parametrize("m,n,LP", [(5000, 200, 16), (1000, 256, 16), (777, 77, 16), (3000, 128, 16),
                                    (4100, 200, 32), (129, 5, 16)])
def test_cols_tc_matches_fp64(fr, m, n, LP):
    """Y = A^T Z on tcgen05 (MN-major A operand, split-K over rows in tensor memory, cluster reduction)."""
    import torch
    rng = np.random.default_rng(7 * m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((m, LP)).astype(np.float32)
    h = fr.Handle(m, n, LP, q=1)
    Y = h.debug_cols_tc(to_gpu(A), LP, B=torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A.T.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A.T).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.max(np.abs(Y - ref) / scale) < 2e-6


@pytest.mark.parametrize("m,n,LP", [(5000, 200, 16), (2000, 64, 32)])
def test_cols_tc_sketch_matches_oracle_omega(fr, m, n, LP):
    """Y = A^T Omega with Omega drawn in-kernel from the Philox stream (Alg. 1 steps 4-5)."""
    from oracle.philox import gaussian_matrix
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)).astype(np.float32)
    h = fr.Handle(m, n, LP, q=1)
    Y = h.debug_cols_tc(to_gpu(A), LP, B=None, seed=99, stream=5).cpu().numpy()
    Om = gaussian_matrix(m, LP, 99, 5)
    ref = A.T.astype(np.float64) @ Om
    scale = np.abs(A.T).astype(np.float64) @ np.abs(Om)
    assert np.max(np.abs(Y - ref) / scale) < 5e-6
